// dslash.cu -- the Wilson-clover operator D = A - kappa H on the whole
// lattice (Eq. 1; the global "Dv" of Alg. 1 line 9 and of Eq. 3).
//
// One thread per site.  Each thread reads its own spinor and clover, then
// for each of the 8 hops the neighbour's spinor and the link, spin-projects
// the neighbour to a two-spin half spinor, multiplies it by U (forward) or
// U^dag (backward) and rebuilds the four-spin result.  All fields are planar
// so that every load of a warp is one contiguous, fully used segment; the
// 8-fold re-reads of neighbour spinors and the 2-fold re-reads of links are
// served by L1/L2, leaving the compulsory traffic (spinor in, links, clover,
// spinor out) for HBM.  Epilogues fuse the residual update and the dot
// products of BiCGStab, so those need no separate pass over memory.
#include <atomic>

#include "device.cuh"
#include "lib.h"
#include "pair.cuh"

namespace qdd {

// D at site x followed by the epilogue; the epilogue's dot products are added
// to part.
template <int P, int EPI>
__device__ __forceinline__ void dslash_site(const DslashArgs &a, long long V, long long x,
                                            typename RealOf<P>::T (&part)[3])
{
    typedef typename RealOf<P>::T T;
    // the epilogue's second vector: in FP16 it is loaded before the stencil
    // so that its latency overlaps the site arithmetic (in FP32/FP64 the
    // registers would cost occupancy).  It is always loaded before out is
    // stored, which the compiler must assume may alias it.
    constexpr bool HAS_Y = EPI != EPI_D;
    constexpr bool EARLY_Y = HAS_Y && P == P16;
    C<T> y[12];
    if constexpr (EARLY_Y) load_spinor<P>(a.y, V, x, y);
    C<T> acc[12];
    if constexpr (P == P16) apply_D_site_f16x2(a.g, a.in, a.U, a.A, (float)a.kappa, x, acc);
    else apply_D_site<P>(a.g, a.in, a.U, a.A, (T)a.kappa, x, acc);
    if constexpr (HAS_Y && !EARLY_Y) load_spinor<P>(a.y, V, x, y);

    if constexpr (EPI == EPI_XMY || EPI == EPI_XMY_NORM) {
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = csub(y[k], acc[k]);
    }
    store_spinor<P>(a.out, V, x, acc);

    if constexpr (EPI == EPI_XMY_NORM) {
        T n2 = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) cnorm_acc(acc[k], n2);
        part[0] += n2;
    } else if constexpr (EPI == EPI_RV || EPI == EPI_TS) {
        T dr = 0, di = 0, n2 = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            // EPI_RV: <y, out> = sum conj(y) out ; EPI_TS: <out, y> = sum conj(out) y
            if constexpr (EPI == EPI_RV) cdot_acc(y[k], acc[k], dr, di);
            else cdot_acc(acc[k], y[k], dr, di);
            cnorm_acc(acc[k], n2);
        }
        part[0] += dr;
        part[1] += di;
        part[2] += n2;
    }
}

template <int P, int EPI, int NT>
__device__ __forceinline__ void dslash_body(DslashArgs a)
{
    typedef typename RealOf<P>::T T;
    constexpr int NRED = (EPI == EPI_XMY_NORM) ? 1 : (EPI == EPI_RV || EPI == EPI_TS) ? 3 : 0;
    const int r = blockIdx.x % a.nrhs;
    const unsigned bid = blockIdx.x / a.nrhs, nblk = gridDim.x / a.nrhs;
    const long long V = a.g.V;
    Scalars *sc = a.sc ? a.sc + r : nullptr;
    if constexpr (EPI == EPI_RV || EPI == EPI_TS) {
        if (sc->status != S_RUN) return;
    }
    a.out = rhs_view<P>(a.out, V, r);
    a.in = rhs_view<P>(a.in, V, r);
    a.y = rhs_view<P>(a.y, V, r);
    T part[3] = {0, 0, 0};

    // one site per thread for the plain epilogues; the reducing ones run on a
    // grid of resident blocks that strides over the lattice, so that each
    // block reduces (and waits at its barrier) once for many sites
    if constexpr (NRED > 0) {
        for (long long x = (long long)bid * NT + threadIdx.x; x < V; x += (long long)nblk * NT)
            dslash_site<P, EPI>(a, V, x, part);
    } else {
        const long long x = (long long)bid * NT + threadIdx.x;
        if (x < V) dslash_site<P, EPI>(a, V, x, part);
    }

    if constexpr (NRED > 0) {
        double red[NRED];
        T pr[NRED];
#pragma unroll
        for (int k = 0; k < NRED; k++) pr[k] = part[k];
        if (grid_sum<NRED, T>(pr, red, rs_partials(a.rs, r), rs_counter(a.rs, r), bid, nblk)) {
            if constexpr (EPI == EPI_XMY_NORM) {
                sc->aux[a.aux_slot] = red[0];
            } else if constexpr (EPI == EPI_RV) {
                const double2 rv = make_double2(red[0], red[1]);
                const double mag2 = rv.x * rv.x + rv.y * rv.y;
                if (!isfinite(mag2) || !isfinite(red[2])) {
                    sc->status = S_NONFINITE;
                } else if (mag2 <= 1e-60 * sc->rhat2 * red[2]) {
                    sc->status = S_BREAK_RV;
                } else {
                    sc->alpha = zdiv(sc->rho, rv);
                }
            } else {
                const double tt = red[2];
                if (!isfinite(tt) || !isfinite(red[0]) || !isfinite(red[1])) {
                    sc->status = S_NONFINITE;
                } else if (tt == 0.0) {
                    sc->status = S_BREAK_TT;
                } else {
                    sc->omega = make_double2(red[0] / tt, red[1] / tt);
                }
            }
        }
    }
}

// FP32 and FP64 keep the compiler's register choice (a register bound there
// makes them spill heavily).  The FP16 kernel works on packed FP32 pairs
// (pair.cuh) with up to 128 registers, two blocks of 256 threads per SM: at 3
// blocks (80 registers) or 5 blocks of 128 threads (96 registers) it measured
// 5-10% slower.
template <int P, int EPI, int NT>
__global__ void __launch_bounds__(NT) dslash_kernel(DslashArgs a)
{
    dslash_body<P, EPI, NT>(a);
}

template <int EPI, int NT>
__global__ void __launch_bounds__(NT, 2) dslash_f16_kernel(DslashArgs a)
{
    dslash_body<P16, EPI, NT>(a);
}

// SMs x resident blocks per SM of one kernel on the current device, queried
// once per device (the values are the same for every caller).
template <int P, int EPI>
static long long resident_blocks(void (*kernel)(DslashArgs), int nt)
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, nt, 0) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        v = sms * (per > 0 ? per : 1);
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <int P, int EPI>
static cudaError_t launch_one(const DslashArgs &a, cudaStream_t st)
{
    constexpr int NT = (P == P64) ? 128 : 256;
    constexpr bool RED = EPI == EPI_XMY_NORM || EPI == EPI_RV || EPI == EPI_TS;
    void (*kernel)(DslashArgs);
    if constexpr (P == P16) kernel = dslash_f16_kernel<EPI, NT>;
    else kernel = dslash_kernel<P, EPI, NT>;
    long long nb = (a.g.V + NT - 1) / NT;
    if (a.nrhs < 1) return cudaErrorInvalidValue;
    if constexpr (RED) {
        const long long cap = resident_blocks<P, EPI>(kernel, NT);
        if (cap > 0 && nb > cap) nb = cap;
        if (nb > a.rs.max_blocks) return cudaErrorInvalidConfiguration;
    }
    kernel<<<(unsigned)(nb * a.nrhs), NT, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <int P>
static cudaError_t launch_prec(int epi, const DslashArgs &a, cudaStream_t st)
{
    switch (epi) {
    case EPI_D: return launch_one<P, EPI_D>(a, st);
    case EPI_XMY: return launch_one<P, EPI_XMY>(a, st);
    case EPI_XMY_NORM: return launch_one<P, EPI_XMY_NORM>(a, st);
    case EPI_RV: return launch_one<P, EPI_RV>(a, st);
    case EPI_TS: return launch_one<P, EPI_TS>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dslash(int prec, int epi, const DslashArgs &a, cudaStream_t st)
{
    if (a.g.V <= 0) return cudaSuccess;
    switch (prec) {
    case P64: return launch_prec<P64>(epi, a, st);
    case P32: return launch_prec<P32>(epi, a, st);
    case P16: return a.nrhs >= 2 ? launch_dslash_mrhs_f16(epi, a, st) : launch_prec<P16>(epi, a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qdd
