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
#include <cstring>

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

// Block bid of the nblk blocks that cover right-hand side r, whose vectors
// `a` already points at (the caller has checked that its solver runs, where
// the epilogue reduces).
template <int P, int EPI, int NT>
__device__ __forceinline__ void dslash_core(const DslashArgs &a, int r, unsigned bid, unsigned nblk)
{
    typedef typename RealOf<P>::T T;
    constexpr int NRED = (EPI == EPI_XMY_NORM) ? 1 : (EPI == EPI_RV || EPI == EPI_TS) ? 3 : 0;
    const long long V = a.g.V;
    Scalars *sc = a.sc ? a.sc + r : nullptr;
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

template <int P, int EPI, int NT>
__device__ __forceinline__ void dslash_body(DslashArgs a)
{
    const int r = blockIdx.x % a.nrhs;
    const unsigned bid = blockIdx.x / a.nrhs, nblk = gridDim.x / a.nrhs;
    const long long V = a.g.V;
    if constexpr (EPI == EPI_RV || EPI == EPI_TS) {
        if (a.sc[r].status != S_RUN) return;
    }
    a.out = rhs_view<P>(a.out, V, r);
    a.in = rhs_view<P>(a.in, V, r);
    a.y = rhs_view<P>(a.y, V, r);
    dslash_core<P, EPI, NT>(a, r, bid, nblk);
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

// D on the lattices of a batch in one launch (a concatenated site range),
// FP16 storage: lattice i owns the blocks first[i] .. first[i+1]-1.  Each
// lattice has one right-hand side; one whose solver no longer runs is
// skipped whole.  The arguments are copied to shared memory once per block.
struct DslashList {
    int n;
    int first[LIST_MAX + 1];
    DslashArgs a[LIST_MAX];
};
static_assert(sizeof(DslashList) <= 32000, "kernel parameter size");

template <int P, int EPI, int NT>
__global__ void __launch_bounds__(NT, 2) dslash_list_kernel(const __grid_constant__ DslashList L)
{
    __shared__ DslashArgs sa;
    const int i = list_member(L.first, L.n);
    const DslashArgs &ga = L.a[i];
    if (ga.sc->status != S_RUN) return;  // uniform over the block
    copy_words(&sa, &ga, sizeof(DslashArgs));
    __syncthreads();
    dslash_core<P, EPI, NT>(sa, 0, blockIdx.x - (unsigned)L.first[i], (unsigned)(L.first[i + 1] - L.first[i]));
}

// SMs x resident blocks per SM of one kernel on the current device, queried
// once per device (the values are the same for every caller).
template <int P, int EPI, typename K>
static long long resident_blocks(K kernel, int nt)
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

// Blocks per lattice: one site per thread for the plain epilogues; for the
// reducing ones the resident grid shared in proportion to the lattice sizes.
template <int P, int EPI>
static cudaError_t launch_list_one(const DslashArgs *as, int n, cudaStream_t st)
{
    constexpr int NT = 256;
    constexpr bool RED = EPI == EPI_XMY_NORM || EPI == EPI_RV || EPI == EPI_TS;
    auto kernel = dslash_list_kernel<P, EPI, NT>;
    if (n < 1 || n > LIST_MAX) return cudaErrorInvalidValue;
    DslashList L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    long long vtot = 0;
    for (int i = 0; i < n; i++) {
        if (as[i].nrhs != 1 || !as[i].sc || as[i].g.V <= 0) return cudaErrorInvalidValue;
        vtot += as[i].g.V;
    }
    const long long cap = RED ? resident_blocks<P, EPI>(kernel, NT) : 0;
    long long total = 0;
    for (int i = 0; i < n; i++) {
        L.a[i] = as[i];
        long long nb = (as[i].g.V + NT - 1) / NT;
        if (RED && cap > 0) {
            const long long share = (cap * as[i].g.V + vtot - 1) / vtot;
            if (nb > share) nb = share;
        }
        if (nb > as[i].rs.max_blocks) nb = as[i].rs.max_blocks;
        L.first[i] = (int)total;
        total += nb < 1 ? 1 : nb;
    }
    L.first[n] = (int)total;
    if (total >= (1LL << 31)) return cudaErrorInvalidConfiguration;
    kernel<<<(unsigned)total, NT, 0, st>>>(L);
    note_launch();
    return cudaGetLastError();
}

// (the epilogues of a BiCGStab iteration preconditioned by K_RAS)
template <int P>
static cudaError_t launch_list_prec(int epi, const DslashArgs *as, int n, cudaStream_t st)
{
    switch (epi) {
    case EPI_XMY: return launch_list_one<P, EPI_XMY>(as, n, st);
    case EPI_RV: return launch_list_one<P, EPI_RV>(as, n, st);
    case EPI_TS: return launch_list_one<P, EPI_TS>(as, n, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dslash_list(int prec, int epi, const DslashArgs *as, int n, cudaStream_t st)
{
    return prec == P16 ? launch_list_prec<P16>(epi, as, n, st) : cudaErrorInvalidValue;
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
