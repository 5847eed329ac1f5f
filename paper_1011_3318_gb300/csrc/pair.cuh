// pair.cuh -- the FP16-storage Wilson-clover operator on packed FP32 pairs.
//
// Blackwell (sm_100 and later) executes two FP32 fused multiply-adds of a
// register pair in one instruction (FFMA2, __ffma2_rn): the same arithmetic
// rate as two scalar FFMAs, half the issue slots.  The FP16 D is bound by
// instruction issue, not by its FP32 pipes, so this file writes its site
// operator (Eq. 1: D = A - kappa H) on pairs of values that undergo identical
// arithmetic:
//
//  * the hops pair spin 0 with spin 1 (and spin 2 with spin 3): the spin
//    projection, the colour matrix-vector product with the link and the
//    reconstruction act on both spins of a chiral half alike.  A spinor is
//    held as real-part pairs R[a] = (psi[s0][a].re, psi[s1][a].re) and
//    imaginary-part pairs I[a] for colours a = 0..2; a link entry enters as
//    a broadcast pair (U.re, U.re).  The off-diagonal X_x and X_y of the
//    projector exchange the two spins: for them the lower half is converted
//    from FP16 straight into the exchanged order, and its reconstruction is
//    written with scalar FMAs.
//  * the clover term pairs its two chiral blocks (spins 0, 1 against spins
//    2, 3): both are packed Hermitian 6x6 matrices of the same shape, so
//    entry p of block 0 and entry p of block 1 form a pair and the product
//    needs no broadcast.
//
// All arithmetic is FP32 with round-to-nearest, as in the scalar operator of
// device.cuh; only the grouping of operations into instructions differs.
//
// Measured limits (32^4, ncu): an FFMA2 occupies both FP32 half-pipes for two
// cycles, while each FP16-to-FP32 conversion occupies only the heavy
// half-pipe, so packing does not relieve the FP32 pipes of the conversions'
// load; it cuts the instructions issued (2353 -> 1765 per site) and the FP16
// D from 92 to 90 us.  What remains is the FP32 pipes (about half the time)
// overlapping with the compulsory DRAM traffic (the other half).
#pragma once

#include <cuda_fp16.h>

#include "device.cuh"



namespace qdd {

typedef float2 f2;

__device__ __forceinline__ f2 pfma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 pmul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 bc2(float x) { return make_float2(x, x); }
__device__ __forceinline__ f2 pneg(f2 a) { return make_float2(-a.x, -a.y); }

// The two halves of a 32-bit word holding one FP16 complex number.
__device__ __forceinline__ float hre(unsigned w) { return __low2float(*reinterpret_cast<const __half2 *>(&w)); }
__device__ __forceinline__ float him(unsigned w) { return __high2float(*reinterpret_cast<const __half2 *>(&w)); }

// The 12 words (one FP16 complex component k = 3 spin + colour each) of the
// FP16 spinor at site i, and its site norm.
__device__ __forceinline__ float load_words16(const SpinorView &f, unsigned v, unsigned i, unsigned (&w)[12])
{
    const uint4 *p = (const uint4 *)f.d;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const uint4 a = p[q * v + i];
        w[4 * q] = a.x;
        w[4 * q + 1] = a.y;
        w[4 * q + 2] = a.z;
        w[4 * q + 3] = a.w;
    }
    return f.n[i];
}

// The 12-real FP16 link U_mu at site i as 18 FP32 reals (row 2 rebuilt as
// conj(row0 x row1)), in the scalar form of device.cuh.
__device__ __forceinline__ void load_link16(const LinkView &u, unsigned v, int mu, unsigned i, C<float> (&U)[9])
{
    const uint2 *p = (const uint2 *)u.d + mu * 3 * v;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const uint2 a = p[q * v + i];
        U[2 * q] = {hre(a.x), him(a.x)};
        U[2 * q + 1] = {hre(a.y), him(a.y)};
    }
    rebuild_row2(U);
}

// One hop on spin pairs: acc += c (1 + s gamma_mu) (x) M psi with s = -1 and
// M = U (forward) or s = +1 and M = U^dag (backward).  psi enters as pairs:
// UR, UI the upper spins (0, 1) of each colour, and DA, DB the lower spins --
// for MU = 2, 3 in the order (spin 2, spin 3) as real and imaginary parts, for
// MU = 0, 1 (whose X exchanges the spins) in the order (spin 3, spin 2).
template <int MU, bool FWD>
__device__ __forceinline__ void hop_core(const f2 (&UR)[3], const f2 (&UI)[3], const f2 (&DA)[3],
                                         const f2 (&DB)[3], const C<float> (&U)[9], float c, f2 (&AUR)[3],
                                         f2 (&AUI)[3], f2 (&ADR)[3], f2 (&ADI)[3])
{
    constexpr float s = FWD ? -1.f : 1.f;
    // h = u + s X_mu d on spin pairs (R: real parts, I: imaginary parts)
    f2 HR[3], HI[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if constexpr (MU == 3) {            // X = 1
            HR[a] = pfma(DA[a], bc2(s), UR[a]);
            HI[a] = pfma(DB[a], bc2(s), UI[a]);
        } else if constexpr (MU == 2) {     // X = diag(i, -i)
            HR[a] = pfma(DB[a], make_float2(-s, s), UR[a]);
            HI[a] = pfma(DA[a], make_float2(s, -s), UI[a]);
        } else if constexpr (MU == 0) {     // X = [[0, i], [i, 0]], d exchanged
            HR[a] = pfma(DB[a], bc2(-s), UR[a]);
            HI[a] = pfma(DA[a], bc2(s), UI[a]);
        } else {                            // X = [[0, -1], [1, 0]], d exchanged
            HR[a] = pfma(DA[a], make_float2(-s, s), UR[a]);
            HI[a] = pfma(DB[a], make_float2(-s, s), UI[a]);
        }
    }
    const f2 cc = bc2(c);
    const float sc = s * c;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        // row a of M h on both spins, M = U or U^dag
        f2 WR, WI;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const C<float> m = FWD ? U[3 * a + b] : C<float>{U[3 * b + a].r, -U[3 * b + a].i};
            const f2 mr = bc2(m.r), mi = bc2(m.i), mn = bc2(-m.i);
            if (b == 0) {
                WR = pmul(mr, HR[0]);
                WI = pmul(mr, HI[0]);
            } else {
                WR = pfma(mr, HR[b], WR);
                WI = pfma(mr, HI[b], WI);
            }
            WR = pfma(mn, HI[b], WR);
            WI = pfma(mi, HR[b], WI);
        }
        // upper half += c w; lower half += c s X^dag w
        AUR[a] = pfma(cc, WR, AUR[a]);
        AUI[a] = pfma(cc, WI, AUI[a]);
        if constexpr (MU == 3) {            // X^dag w = w
            ADR[a] = pfma(bc2(sc), WR, ADR[a]);
            ADI[a] = pfma(bc2(sc), WI, ADI[a]);
        } else if constexpr (MU == 2) {     // X^dag w = (-i w0, i w1)
            ADR[a] = pfma(make_float2(sc, -sc), WI, ADR[a]);
            ADI[a] = pfma(make_float2(-sc, sc), WR, ADI[a]);
        } else if constexpr (MU == 0) {     // X^dag w = (-i w1, -i w0)
            ADR[a].x = fmaf(sc, WI.y, ADR[a].x);
            ADR[a].y = fmaf(sc, WI.x, ADR[a].y);
            ADI[a].x = fmaf(-sc, WR.y, ADI[a].x);
            ADI[a].y = fmaf(-sc, WR.x, ADI[a].y);
        } else {                            // X^dag w = (w1, -w0)
            ADR[a].x = fmaf(sc, WR.y, ADR[a].x);
            ADR[a].y = fmaf(-sc, WR.x, ADR[a].y);
            ADI[a].x = fmaf(sc, WI.y, ADI[a].x);
            ADI[a].y = fmaf(-sc, WI.x, ADI[a].y);
        }
    }
}

// The same hop with psi given as the 12 FP16 words of the neighbour (one
// complex component k = 3 spin + colour each): the lower spins are converted
// straight into the order hop_core expects.
template <int MU, bool FWD>
__device__ __forceinline__ void hop_pair16(const unsigned (&w)[12], const C<float> (&U)[9], float c, f2 (&AUR)[3],
                                           f2 (&AUI)[3], f2 (&ADR)[3], f2 (&ADI)[3])
{
    f2 UR[3], UI[3], DA[3], DB[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        UR[a] = make_float2(hre(w[a]), hre(w[3 + a]));
        UI[a] = make_float2(him(w[a]), him(w[3 + a]));
        if constexpr (MU >= 2) {
            DA[a] = make_float2(hre(w[6 + a]), hre(w[9 + a]));
            DB[a] = make_float2(him(w[6 + a]), him(w[9 + a]));
        } else {
            DA[a] = make_float2(hre(w[9 + a]), hre(w[6 + a]));
            DB[a] = make_float2(him(w[9 + a]), him(w[6 + a]));
        }
    }
    hop_core<MU, FWD>(UR, UI, DA, DB, U, c, AUR, AUI, ADR, ADI);
}

// The data of both hops in direction MU at site x: the two neighbours' FP16
// words and norms and the raw FP16 links (forward: U_mu(x); backward:
// U_mu(x - mu)), with the hop coefficients.
struct HopData {
    unsigned wf[12], wb[12];
    uint2 lf[3], lb[3];
    float cf, cb;
};

template <int MU>
__device__ __forceinline__ void hop_load16(const Geom &g, const SpinorView &in, const LinkView &Ul, unsigned x,
                                           const int c[4], float mk, HopData &h)
{
    const unsigned v = (unsigned)g.V;
    const unsigned xf = (unsigned)fwd_site(g, x, c, MU), xb = (unsigned)bwd_site(g, x, c, MU);
    const float sf = (c[MU] == g.L[MU] - 1 && g.bc[MU] < 0) ? -mk : mk;
    const float sb = (c[MU] == 0 && g.bc[MU] < 0) ? -mk : mk;
    h.cf = sf * load_words16(in, v, xf, h.wf);
    h.cb = sb * load_words16(in, v, xb, h.wb);
    const uint2 *p = (const uint2 *)Ul.d + MU * 3 * v;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        h.lf[q] = p[q * v + x];
        h.lb[q] = p[q * v + xb];
    }
}

__device__ __forceinline__ void link_from_words(const uint2 (&l)[3], C<float> (&U)[9])
{
#pragma unroll
    for (int q = 0; q < 3; q++) {
        U[2 * q] = {hre(l[q].x), him(l[q].x)};
        U[2 * q + 1] = {hre(l[q].y), him(l[q].y)};
    }
    rebuild_row2(U);
}

template <int MU>
__device__ __forceinline__ void hop_apply16(const HopData &h, f2 (&AUR)[3], f2 (&AUI)[3], f2 (&ADR)[3], f2 (&ADI)[3])
{
    {
        C<float> U[9];
        link_from_words(h.lf, U);
        hop_pair16<MU, true>(h.wf, U, h.cf, AUR, AUI, ADR, ADI);
    }
    {
        C<float> U[9];
        link_from_words(h.lb, U);
        hop_pair16<MU, false>(h.wb, U, h.cb, AUR, AUI, ADR, ADI);
    }
}

// Both hops in direction MU from FP16 fields in global memory.
template <int MU>
__device__ __forceinline__ void hop_dir16(const Geom &g, const SpinorView &in, const LinkView &Ul, unsigned x,
                                          const int c[4], float mk, f2 (&AUR)[3], f2 (&AUI)[3], f2 (&ADR)[3],
                                          f2 (&ADI)[3])
{
    HopData h;
    hop_load16<MU>(g, in, Ul, x, c, mk, h);
    hop_apply16<MU>(h, AUR, AUI, ADR, ADI);
}

// acc += sc A psi (INIT: acc = sc A psi) for the FP16 clover planes p (plane
// k of the site at p[k * v + i]; global or shared memory) and psi as chiral
// pairs SR[j] = (psi[j].re, psi[6 + j].re), SI[j] likewise, j = 3 spin +
// colour: the two chiral 6x6 blocks as pairs (block 0, block 1).  Word m of
// the FP16 clover holds entry m of both blocks, so one conversion per half
// gives the pair, and the entries stream in storage order: each is applied to
// both rows it belongs to (an off-diagonal entry L_rj, r > j, gives L_rj psi_j
// to row r and conj(L_rj) psi_r to row j).
template <bool INIT>
__device__ __forceinline__ void clover_core(const uint4 *p, unsigned v, unsigned i, const f2 (&SR)[6],
                                            const f2 (&SI)[6], float sc, f2 (&AUR)[3], f2 (&AUI)[3], f2 (&ADR)[3],
                                            f2 (&ADI)[3])
{
    f2 OR[6], OI[6];
    f2 e[36];   // entry m of both blocks (the compiler keeps only the live ones)
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const uint4 q = p[k * v + i];
        e[4 * k] = make_float2(hre(q.x), him(q.x));
        e[4 * k + 1] = make_float2(hre(q.y), him(q.y));
        e[4 * k + 2] = make_float2(hre(q.z), him(q.z));
        e[4 * k + 3] = make_float2(hre(q.w), him(q.w));
    }
#pragma unroll
    for (int r = 0; r < 6; r++) {
        OR[r] = pmul(e[r], SR[r]);
        OI[r] = pmul(e[r], SI[r]);
    }
#pragma unroll
    for (int r = 1; r < 6; r++)
#pragma unroll
        for (int j = 0; j < r; j++) {
            const int off = cl_off(r, j);
            const f2 lr = e[off], li = e[off + 1];
            // row r: += L psi_j
            OR[r] = pfma(lr, SR[j], OR[r]);
            OR[r] = pfma(pneg(li), SI[j], OR[r]);
            OI[r] = pfma(lr, SI[j], OI[r]);
            OI[r] = pfma(li, SR[j], OI[r]);
            // row j: += conj(L) psi_r
            OR[j] = pfma(lr, SR[r], OR[j]);
            OR[j] = pfma(li, SI[r], OR[j]);
            OI[j] = pfma(lr, SI[r], OI[j]);
            OI[j] = pfma(pneg(li), SR[r], OI[j]);
        }
    // block 0 -> spins 0, 1 (upper pairs); block 1 -> spins 2, 3 (lower pairs)
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if constexpr (INIT) {
            AUR[a] = make_float2(sc * OR[a].x, sc * OR[3 + a].x);
            AUI[a] = make_float2(sc * OI[a].x, sc * OI[3 + a].x);
            ADR[a] = make_float2(sc * OR[a].y, sc * OR[3 + a].y);
            ADI[a] = make_float2(sc * OI[a].y, sc * OI[3 + a].y);
        } else {
            AUR[a].x = fmaf(sc, OR[a].x, AUR[a].x);
            AUR[a].y = fmaf(sc, OR[3 + a].x, AUR[a].y);
            AUI[a].x = fmaf(sc, OI[a].x, AUI[a].x);
            AUI[a].y = fmaf(sc, OI[3 + a].x, AUI[a].y);
            ADR[a].x = fmaf(sc, OR[a].y, ADR[a].x);
            ADR[a].y = fmaf(sc, OR[3 + a].y, ADR[a].y);
            ADI[a].x = fmaf(sc, OI[a].y, ADI[a].x);
            ADI[a].y = fmaf(sc, OI[3 + a].y, ADI[a].y);
        }
    }
}

// The clover term for psi given as the 12 FP16 words of the site.
template <bool INIT>
__device__ __forceinline__ void clover_pair16(const CloverView &A, unsigned v, unsigned i, const unsigned (&w)[12],
                                              float sc, f2 (&AUR)[3], f2 (&AUI)[3], f2 (&ADR)[3], f2 (&ADI)[3])
{
    f2 SR[6], SI[6];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        SR[j] = make_float2(hre(w[j]), hre(w[6 + j]));
        SI[j] = make_float2(him(w[j]), him(w[6 + j]));
    }
    clover_core<INIT>((const uint4 *)A.d, v, i, SR, SI, sc, AUR, AUI, ADR, ADI);
}

// (D in)(x) for FP16 fields on packed pairs; the result in the scalar
// component order of device.cuh (acc[3 spin + colour]).
__device__ __forceinline__ void apply_D_site_f16x2(const Geom &g, const SpinorView &in, const LinkView &Ul,
                                                   const CloverView &A, float kappa, long long xl, C<float> (&acc)[12])
{
    const unsigned x = (unsigned)xl, v = (unsigned)g.V;
    int c[4];
    site_coords(g, xl, c);
    const float mk = -kappa;
    f2 AUR[3], AUI[3], ADR[3], ADI[3];
    // the clover term first, as the accumulators' initial value: its words
    // are then never live together with the hop accumulators (fewer
    // registers; loading each direction's data before the previous
    // direction's arithmetic measured no faster)
    {
        unsigned w[12];
        const float ns = load_words16(in, v, x, w);
        clover_pair16<true>(A, v, x, w, ns * A.n[x], AUR, AUI, ADR, ADI);
    }
    hop_dir16<0>(g, in, Ul, x, c, mk, AUR, AUI, ADR, ADI);
    hop_dir16<1>(g, in, Ul, x, c, mk, AUR, AUI, ADR, ADI);
    hop_dir16<2>(g, in, Ul, x, c, mk, AUR, AUI, ADR, ADI);
    hop_dir16<3>(g, in, Ul, x, c, mk, AUR, AUI, ADR, ADI);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        acc[a] = {AUR[a].x, AUI[a].x};
        acc[3 + a] = {AUR[a].y, AUI[a].y};
        acc[6 + a] = {ADR[a].x, ADI[a].x};
        acc[9 + a] = {ADR[a].y, ADI[a].y};
    }
}

}  // namespace qdd
