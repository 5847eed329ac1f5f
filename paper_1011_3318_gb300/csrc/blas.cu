// blas.cu -- fused vector kernels of the right-preconditioned BiCGStab
// (Eq. 3) and of the FP64 defect correction around it (Sec. 3).
//
// The solver scalars (rho, alpha, omega, beta, |r|^2) live on the device.
// Each reduction ends with the last-block pattern of grid_sum, whose final
// block derives the next scalar (so no kernel recomputes it per thread and
// no host round trip is needed inside an iteration).  Kernels of a solver
// iteration return at once when the status is no longer "running", which
// lets the host enqueue several iterations ahead of the convergence check.
#include <cstring>

#include "device.cuh"
#include "df64.cuh"
#include "lib.h"

namespace qdd {

constexpr int BLAS_NT = 256;

template <typename T>
__device__ __forceinline__ void zero12(C<T> (&a)[12])
{
#pragma unroll
    for (int k = 0; k < 12; k++) a[k] = {0, 0};
}

template <int P, int OP>
__global__ void __launch_bounds__(BLAS_NT) blas_kernel(BlasArgs a)
{
    typedef typename RealOf<P>::T T;
    constexpr int NRED = (OP == B_INIT || OP == B_NORM || OP == B_RESTART) ? 1 : 0;
    const int r = blockIdx.x % a.nrhs;
    const unsigned bid = blockIdx.x / a.nrhs, nblk = gridDim.x / a.nrhs;
    Scalars *sc = a.sc ? a.sc + r : nullptr;
    if constexpr (OP == B_P || OP == B_S) {
        if (sc->status != S_RUN) return;
    }
    if constexpr (OP == B_RESTART) {
        // restart only the right-hand sides whose BiCGStab broke down
        if (sc->status != S_BREAK_RV && sc->status != S_BREAK_TT) return;
    }
    const long long V = a.V;
#pragma unroll
    for (int i = 0; i < 8; i++) a.f[i] = rhs_view<P>(a.f[i], V, r);
    T part[NRED > 0 ? NRED : 1];
#pragma unroll
    for (int k = 0; k < (NRED > 0 ? NRED : 1); k++) part[k] = 0;

    // coefficients read once per thread from the device scalars
    C<T> c1 = {0, 0}, c2 = {0, 0};
    if constexpr (OP == B_P) {
        c1 = {(T)sc->beta.x, (T)sc->beta.y};
        c2 = {(T)sc->omega.x, (T)sc->omega.y};
    } else if constexpr (OP == B_S) {
        c1 = {(T)sc->alpha.x, (T)sc->alpha.y};
    }

    for (long long x = (long long)bid * BLAS_NT + threadIdx.x; x < V; x += (long long)nblk * BLAS_NT) {
        if constexpr (OP == B_INIT) {
            C<T> b[12], z[12];
            load_spinor<P>(a.f[0], V, x, b);
            zero12(z);
            store_spinor<P>(a.f[1], V, x, b);
            store_spinor<P>(a.f[2], V, x, b);
            store_spinor<P>(a.f[3], V, x, z);
            store_spinor<P>(a.f[4], V, x, z);
            store_spinor<P>(a.f[5], V, x, z);
            T n2 = 0;
#pragma unroll
            for (int k = 0; k < 12; k++) cnorm_acc(b[k], n2);
            part[0] += n2;
        } else if constexpr (OP == B_P) {
            C<T> p[12], r[12], v[12];
            load_spinor<P>(a.f[0], V, x, p);
            load_spinor<P>(a.f[1], V, x, r);
            load_spinor<P>(a.f[2], V, x, v);
#pragma unroll
            for (int k = 0; k < 12; k++) p[k] = cfma(c1, cfma(cneg(c2), v[k], p[k]), r[k]);
            store_spinor<P>(a.f[0], V, x, p);
        } else if constexpr (OP == B_S) {
            C<T> r[12], v[12];
            load_spinor<P>(a.f[1], V, x, r);
            load_spinor<P>(a.f[2], V, x, v);
#pragma unroll
            for (int k = 0; k < 12; k++) r[k] = cfma(cneg(c1), v[k], r[k]);
            store_spinor<P>(a.f[0], V, x, r);
        } else if constexpr (OP == B_NORM) {
            C<T> f[12];
            load_spinor<P>(a.f[0], V, x, f);
            T n2 = 0;
#pragma unroll
            for (int k = 0; k < 12; k++) cnorm_acc(f[k], n2);
            part[0] += n2;
        } else if constexpr (OP == B_COPY) {
            C<T> f[12];
            load_spinor<P>(a.f[1], V, x, f);
            store_spinor<P>(a.f[0], V, x, f);
        } else if constexpr (OP == B_ZERO) {
            C<T> z[12];
            zero12(z);
            store_spinor<P>(a.f[0], V, x, z);
        } else if constexpr (OP == B_AXPY) {
            C<T> f[12], g[12];
            load_spinor<P>(a.f[0], V, x, f);
            load_spinor<P>(a.f[1], V, x, g);
#pragma unroll
            for (int k = 0; k < 12; k++) f[k] = cadd(f[k], g[k]);
            store_spinor<P>(a.f[0], V, x, f);
        } else if constexpr (OP == B_RESTART) {
            C<T> r[12], z[12];
            load_spinor<P>(a.f[1], V, x, r);
            zero12(z);
            store_spinor<P>(a.f[0], V, x, r);
            store_spinor<P>(a.f[2], V, x, z);
            store_spinor<P>(a.f[3], V, x, z);
            T n2 = 0;
#pragma unroll
            for (int k = 0; k < 12; k++) cnorm_acc(r[k], n2);
            part[0] += n2;
        }
    }

    if constexpr (NRED > 0) {
        double red[NRED];
        if (grid_sum<NRED, T>(part, red, rs_partials(a.rs, r), rs_counter(a.rs, r), bid, nblk)) {
            if constexpr (OP == B_INIT) {
                sc->rho = make_double2(red[0], 0.0);
                sc->alpha = sc->omega = sc->beta = make_double2(1.0, 0.0);
                sc->rr = red[0];
                sc->rhat2 = red[0];
                // relative tolerance^2: from the arguments, or per right-hand side from aux[7]
                sc->tol2 = (a.tol2_rel >= 0 ? a.tol2_rel : sc->aux[7]) * red[0];
                sc->iter = 0;
                sc->status = isfinite(red[0]) ? (red[0] <= sc->tol2 ? S_CONVERGED : S_RUN) : S_NONFINITE;
                if (!((a.active >> r) & 1ull)) sc->status = S_CONVERGED;
            } else if constexpr (OP == B_NORM) {
                sc->aux[a.aux_slot] = red[0];
            } else if constexpr (OP == B_RESTART) {
                sc->rho = make_double2(red[0], 0.0);
                sc->alpha = sc->omega = sc->beta = make_double2(1.0, 0.0);
                sc->rhat2 = red[0];
                sc->status = isfinite(red[0]) ? S_RUN : S_NONFINITE;
            }
        }
    }
}

// x += alpha phat + omega shat ; r = s - omega t ; then rho' = <rhat, r>,
// |r|^2 and beta = (rho'/rho)(alpha/omega).  f = {x, phat, shat, r, s, t, rhat}.
// Block bid of the nblk blocks of right-hand side r, whose vectors `a`
// already points at and whose solver runs.
template <int P>
__device__ __forceinline__ void bicg_xr_core(const BlasArgs &a, int r, unsigned bid, unsigned nblk)
{
    typedef typename RealOf<P>::T T;
    Scalars *sc = a.sc + r;
    const long long V = a.V;
    const C<T> al = {(T)sc->alpha.x, (T)sc->alpha.y};
    const C<T> om = {(T)sc->omega.x, (T)sc->omega.y};
    T part[3] = {0, 0, 0};
    for (long long x = (long long)bid * BLAS_NT + threadIdx.x; x < V; x += (long long)nblk * BLAS_NT) {
        C<T> xx[12], ph[12], sh[12];
        load_spinor<P>(a.f[0], V, x, xx);
        load_spinor<P>(a.f[1], V, x, ph);
        load_spinor<P>(a.f[2], V, x, sh);
#pragma unroll
        for (int k = 0; k < 12; k++) xx[k] = cfma(om, sh[k], cfma(al, ph[k], xx[k]));
        store_spinor<P>(a.f[0], V, x, xx);
        C<T> s[12], t[12], rh[12];
        load_spinor<P>(a.f[4], V, x, s);
        load_spinor<P>(a.f[5], V, x, t);
        load_spinor<P>(a.f[6], V, x, rh);
        T dr = 0, di = 0, n2 = 0;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            s[k] = cfma(cneg(om), t[k], s[k]);
            cdot_acc(rh[k], s[k], dr, di);
            cnorm_acc(s[k], n2);
        }
        store_spinor<P>(a.f[3], V, x, s);
        part[0] += dr;
        part[1] += di;
        part[2] += n2;
    }
    double red[3];
    if (grid_sum<3, T>(part, red, rs_partials(a.rs, r), rs_counter(a.rs, r), bid, nblk)) {
        const double2 rn = make_double2(red[0], red[1]);
        if (!isfinite(red[0]) || !isfinite(red[1]) || !isfinite(red[2])) {
            sc->status = S_NONFINITE;
            return;
        }
        sc->beta = zmul(zdiv(rn, sc->rho), zdiv(sc->alpha, sc->omega));
        sc->rho = rn;
        sc->rr = red[2];
        sc->iter += 1;
        if (red[2] <= sc->tol2) sc->status = S_CONVERGED;
    }
}

template <int P>
__global__ void __launch_bounds__(BLAS_NT) bicg_xr_kernel(BlasArgs a)
{
    const int r = blockIdx.x % a.nrhs;
    const unsigned bid = blockIdx.x / a.nrhs, nblk = gridDim.x / a.nrhs;
    if (a.sc[r].status != S_RUN) return;
#pragma unroll
    for (int i = 0; i < 8; i++) a.f[i] = rhs_view<P>(a.f[i], a.V, r);
    bicg_xr_core<P>(a, r, bid, nblk);
}

// B_XR on the lattices of a batch in one launch: lattice i owns the blocks
// first[i] .. first[i+1]-1 and has one right-hand side; one whose solver no
// longer runs is skipped.
struct BlasList {
    int n;
    int first[LIST_MAX + 1];
    BlasArgs a[LIST_MAX];
};
static_assert(sizeof(BlasList) <= 32000, "kernel parameter size");

template <int P>
__global__ void __launch_bounds__(BLAS_NT) bicg_xr_list_kernel(const __grid_constant__ BlasList L)
{
    __shared__ BlasArgs sa;
    const int i = list_member(L.first, L.n);
    const BlasArgs &ga = L.a[i];
    if (ga.sc->status != S_RUN) return;  // uniform over the block
    copy_words(&sa, &ga, sizeof(BlasArgs));
    __syncthreads();
    bicg_xr_core<P>(sa, 0, blockIdx.x - (unsigned)L.first[i], (unsigned)(L.first[i + 1] - L.first[i]));
}

static int blas_blocks(long long V, int max_blocks)
{
    long long nb = (V + BLAS_NT - 1) / BLAS_NT;
    long long cap = 152LL * 8;  // 8 resident blocks of 256 threads on each of the 152 SMs
    if (nb > cap) nb = cap;
    if (nb > max_blocks) nb = max_blocks;
    return (int)(nb < 1 ? 1 : nb);
}

template <int P>
static cudaError_t launch_blas_p(int op, const BlasArgs &a, cudaStream_t st)
{
    if (a.nrhs < 1) return cudaErrorInvalidValue;
    const int nb = blas_blocks(a.V, a.rs.max_blocks) * a.nrhs;
    switch (op) {
    case B_INIT: blas_kernel<P, B_INIT><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_P: blas_kernel<P, B_P><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_S: blas_kernel<P, B_S><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_XR: bicg_xr_kernel<P><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_NORM: blas_kernel<P, B_NORM><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_COPY: blas_kernel<P, B_COPY><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_ZERO: blas_kernel<P, B_ZERO><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_RESTART: blas_kernel<P, B_RESTART><<<nb, BLAS_NT, 0, st>>>(a); break;
    case B_AXPY: blas_kernel<P, B_AXPY><<<nb, BLAS_NT, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

// The resident grid (blas_blocks) shared by the lattices in proportion to
// their sizes.
template <int P>
static cudaError_t launch_xr_list(const BlasArgs *as, int n, cudaStream_t st)
{
    if (n < 1 || n > LIST_MAX) return cudaErrorInvalidValue;
    BlasList L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    long long vtot = 0;
    for (int i = 0; i < n; i++) {
        if (as[i].nrhs != 1 || !as[i].sc || as[i].V <= 0) return cudaErrorInvalidValue;
        vtot += as[i].V;
    }
    const long long cap = 152LL * 8;
    long long total = 0;
    for (int i = 0; i < n; i++) {
        L.a[i] = as[i];
        long long nb = blas_blocks(as[i].V, as[i].rs.max_blocks);
        const long long share = (cap * as[i].V + vtot - 1) / vtot;
        if (nb > share) nb = share;
        L.first[i] = (int)total;
        total += nb < 1 ? 1 : nb;
    }
    L.first[n] = (int)total;
    bicg_xr_list_kernel<P><<<(unsigned)total, BLAS_NT, 0, st>>>(L);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_blas_list(int prec, int op, const BlasArgs *as, int n, cudaStream_t st)
{
    if (op != B_XR || prec != P16) return cudaErrorInvalidValue;
    return launch_xr_list<P16>(as, n, st);
}

cudaError_t launch_blas(int prec, int op, const BlasArgs &a, cudaStream_t st)
{
    switch (prec) {
    case P64: return launch_blas_p<P64>(op, a, st);
    case P32: return launch_blas_p<P32>(op, a, st);
    case P16: return launch_blas_p<P16>(op, a, st);
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- precision changes
template <int PD>
__global__ void __launch_bounds__(BLAS_NT) convert_scaled_kernel(long long V, SpinorView dst, SpinorView src64,
                                                                 const Scalars *sc, int slot, int nrhs)
{
    typedef typename RealOf<PD>::T T;
    const int r = blockIdx.x % nrhs;
    const unsigned bid = blockIdx.x / nrhs, nblk = gridDim.x / nrhs;
    dst = rhs_view<PD>(dst, V, r);
    src64 = rhs_view<P64>(src64, V, r);
    // 1/|r| once per block (an FP64 division and square root are long
    // sequences on this GPU's FP64 pipe)
    __shared__ double s_inv;
    if (threadIdx.x == 0) {
        const double n2 = sc[r].aux[slot];
        s_inv = n2 > 0 ? 1.0 / sqrt(n2) : 0.0;
    }
    __syncthreads();
    const double inv = s_inv;
    const float invf = (float)inv;
    // values in the normal float range are converted in integer arithmetic
    // and scaled in FP32 (|value * inv| <= 1); others are scaled in FP64 first
    auto cvt = [&](double v) -> T {
        if constexpr (PD == P64) return (T)(v * inv);
        else {
            const int e = dexp(v);
            return (e >= 897 && e <= 1150 && invf > 0.f && invf < 3.0e38f) ? d2f_rn(v) * invf
                                                                             : __double2float_rn(v * inv);
        }
    };
    for (long long x = (long long)bid * BLAS_NT + threadIdx.x; x < V; x += (long long)nblk * BLAS_NT) {
        C<double> s[12];
        load_spinor<P64>(src64, V, x, s);
        C<T> d[12];
#pragma unroll
        for (int k = 0; k < 12; k++) d[k] = {cvt(s[k].r), cvt(s[k].i)};
        store_spinor<PD>(dst, V, x, d);
    }
}

template <int PS>
__global__ void __launch_bounds__(BLAS_NT) accum_scaled_kernel(long long V, SpinorView phi64, SpinorView xs,
                                                               const Scalars *sc, int slot, int nrhs)
{
    typedef typename RealOf<PS>::T T;
    const int r = blockIdx.x % nrhs;
    const unsigned bid = blockIdx.x / nrhs, nblk = gridDim.x / nrhs;
    phi64 = rhs_view<P64>(phi64, V, r);
    xs = rhs_view<PS>(xs, V, r);
    __shared__ double s_sc;
    if (threadIdx.x == 0) s_sc = sqrt(sc[r].aux[slot]);  // once per block
    __syncthreads();
    const double sc_ = s_sc;
    for (long long x = (long long)bid * BLAS_NT + threadIdx.x; x < V; x += (long long)nblk * BLAS_NT) {
        C<double> p[12];
        C<T> e[12];
        load_spinor<P64>(phi64, V, x, p);
        load_spinor<PS>(xs, V, x, e);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            if constexpr (PS == P64) {
                p[k].r += sc_ * (double)e[k].r;
                p[k].i += sc_ * (double)e[k].i;
            } else {  // exact widening in integer arithmetic
                p[k].r = fma(sc_, f2d(e[k].r), p[k].r);
                p[k].i = fma(sc_, f2d(e[k].i), p[k].i);
            }
        }
        store_spinor<P64>(phi64, V, x, p);
    }
}

template <int PD, int PS>
__global__ void __launch_bounds__(BLAS_NT) convert_kernel(long long V, SpinorView dst, SpinorView src, int nrhs)
{
    typedef typename RealOf<PS>::T TS;
    typedef typename RealOf<PD>::T TD;
    const int r = blockIdx.x % nrhs;
    const unsigned bid = blockIdx.x / nrhs, nblk = gridDim.x / nrhs;
    dst = rhs_view<PD>(dst, V, r);
    src = rhs_view<PS>(src, V, r);
    for (long long x = (long long)bid * BLAS_NT + threadIdx.x; x < V; x += (long long)nblk * BLAS_NT) {
        C<TS> s[12];
        load_spinor<PS>(src, V, x, s);
        C<TD> d[12];
#pragma unroll
        for (int k = 0; k < 12; k++) d[k] = {(TD)s[k].r, (TD)s[k].i};
        store_spinor<PD>(dst, V, x, d);
    }
}

cudaError_t launch_convert_scaled(long long V, int prec, SpinorView dst, SpinorView src64, const Scalars *sc,
                                  int slot, int nrhs, cudaStream_t st)
{
    const int nb = blas_blocks(V, 1 << 30) * nrhs;
    if (prec == P64) convert_scaled_kernel<P64><<<nb, BLAS_NT, 0, st>>>(V, dst, src64, sc, slot, nrhs);
    else if (prec == P32) convert_scaled_kernel<P32><<<nb, BLAS_NT, 0, st>>>(V, dst, src64, sc, slot, nrhs);
    else convert_scaled_kernel<P16><<<nb, BLAS_NT, 0, st>>>(V, dst, src64, sc, slot, nrhs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_accum_scaled(long long V, int prec, SpinorView phi64, SpinorView x, const Scalars *sc, int slot,
                                int nrhs, cudaStream_t st)
{
    const int nb = blas_blocks(V, 1 << 30) * nrhs;
    if (prec == P64) accum_scaled_kernel<P64><<<nb, BLAS_NT, 0, st>>>(V, phi64, x, sc, slot, nrhs);
    else if (prec == P32) accum_scaled_kernel<P32><<<nb, BLAS_NT, 0, st>>>(V, phi64, x, sc, slot, nrhs);
    else accum_scaled_kernel<P16><<<nb, BLAS_NT, 0, st>>>(V, phi64, x, sc, slot, nrhs);
    note_launch();
    return cudaGetLastError();
}

template <int PD>
static cudaError_t convert_from(long long V, SpinorView dst, int ps, SpinorView src, int nb, int nrhs,
                                cudaStream_t st)
{
    if (ps == P64) convert_kernel<PD, P64><<<nb, BLAS_NT, 0, st>>>(V, dst, src, nrhs);
    else if (ps == P32) convert_kernel<PD, P32><<<nb, BLAS_NT, 0, st>>>(V, dst, src, nrhs);
    else convert_kernel<PD, P16><<<nb, BLAS_NT, 0, st>>>(V, dst, src, nrhs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_convert(long long V, int pd, SpinorView dst, int ps, SpinorView src, int nrhs, cudaStream_t st)
{
    const int nb = blas_blocks(V, 1 << 30) * nrhs;
    if (pd == P64) return convert_from<P64>(V, dst, ps, src, nb, nrhs, st);
    if (pd == P32) return convert_from<P32>(V, dst, ps, src, nb, nrhs, st);
    return convert_from<P16>(V, dst, ps, src, nb, nrhs, st);
}

}  // namespace qdd
