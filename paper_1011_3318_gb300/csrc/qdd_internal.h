// qdd_internal.h -- types shared by the library's translation units.
//
// Internal GPU layouts (all "planar": one plane of V elements per vector
// component group, so that thread x of a warp reads element x of each plane
// and every load instruction is fully coalesced):
//
//   spinor F64  double2[12][V]     12 complex, index k = 3*spin + colour
//   spinor F32  float4 [6][V]      plane p holds complex k = 2p, 2p+1
//   spinor F16  uint4  [3][V]      8 halves (4 complex) per plane, values
//               + float[V] norm    divided by the site's max |component|
//   links  F64  double2[4][9][V]   full 3x3 per direction (18 reals)
//   links  F32  float4 [4][3][V]   rows 0 and 1 only (12 reals); row 2 is
//   links  F16  uint2  [4][3][V]   rebuilt as conj(row0 x row1)
//   clover F64  double2[36][V]     two Hermitian 6x6 chiral blocks packed as
//   clover F32  float4 [18][V]     6 real diagonals + 15 complex lower
//   clover F16  uint4  [9][V]      off-diagonals (i > j, row-major) each,
//               + float[V] norm    72 reals per site; in FP16, word m holds
//                                  entry m of block 0 (low half) and entry m
//                                  of block 1 (high half)
//
// The clover blocks act on complex components k = 0..5 (spins 0, 1) and
// k = 6..11 (spins 2, 3): in the DeGrand-Rossi basis gamma_5 = diag(1,1,-1,-1)
// and every sigma_{mu nu} is block diagonal in chirality.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qdd.h"

namespace qdd {

enum Prec { P64 = 0, P32 = 1, P16 = 2 };

struct Geom {
    int L[4];
    int bc[4];
    long long stride[4];
    long long V;
};

// Multiplier and shift of the division by d (1 <= d <= 2^30) for numerators
// below 2^31: m = ceil(2^p / d), p = 31 + ceil(log2 d), shift p - 32.
inline void division_magic(int d, unsigned *m, int *sh)
{
    int l = 0;
    while ((1LL << l) < d) l++;
    const int p = 31 + l;
    *m = d >= 2 ? (unsigned)(((1ULL << p) + (unsigned long long)d - 1) / (unsigned long long)d) : 0u;
    *sh = d >= 2 ? p - 32 : 0;
}

// A spinor field in the internal layout of its precision.
struct SpinorView {
    void *d;
    float *n;  // F16 norms
};

struct LinkView {
    const void *d;
};

struct CloverView {
    const void *d;
    const float *n;  // F16 norms
};

// Extended-domain geometry of the RAS decomposition (Sec. 2, Sec. 4).
struct DomainGeom {
    int b[4];    // bulk block
    int e[4];    // extended length (b + 2s, or L when b = L)
    int sh[4];   // offset of the bulk inside the extended domain (s or 0)
    int nb[4];   // blocks per direction
    int ndom;
    int nloc;    // sites in an extended domain
    // division by nb[mu] and e[mu] of numerators below 2^31 as a multiply-high
    // and a shift (Granlund and Montgomery): n / d = umulhi(n, m) >> sh for
    // d >= 2, with m = ceil(2^p / d), p = 31 + ceil(log2 d), sh = p - 32
    unsigned nb_m[4], e_m[4];
    int nb_sh[4], e_sh[4];
};

// Solver scalars kept on the device so that an iteration needs no host
// round trip (complex numbers as double2).
struct Scalars {
    double2 rho;     // <rhat, r> of the current iterate
    double2 alpha;
    double2 omega;
    double2 beta;
    double rr;       // |r|^2 of the recursive residual
    double rhat2;    // |rhat|^2
    double tol2;     // stop when rr <= tol2
    int status;      // 0 running, 1 converged, 2 breakdown <rhat,v>, 3 breakdown <t,t>, 4 non-finite
    int iter;
    double aux[8];   // plain reduction results (norms)
};

// S_TIMEOUT: a bounded device-side wait gave up (reported as QDD_ERR_TIMEOUT).
enum ScalarStatus { S_RUN = 0, S_CONVERGED = 1, S_BREAK_RV = 2, S_BREAK_TT = 3, S_NONFINITE = 4, S_TIMEOUT = 5 };

// Grid-reduction scratch: per-block partial sums and the arrival counter of
// the last-block pattern.
struct ReduceScratch {
    double *partials;
    unsigned int *counter;
    int max_blocks;
};

}  // namespace qdd
