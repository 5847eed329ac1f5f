// dslash_mrhs.cu -- the FP16-storage Wilson-clover D (Eq. 1) on two
// right-hand sides at once.
//
// A lattice with several right-hand sides applies the same links and clover
// to every one of them.  One thread takes one site and two right-hand sides
// (ra, rb): it loads and decodes each link (FP16 rows 0 and 1, row 2 rebuilt)
// and the clover block entries once, and applies them to both spinors.  The
// two right-hand sides undergo identical arithmetic, so every FP32 operation
// is one packed instruction on the pair (value for ra, value for rb)
// (FFMA2, sm_100 and later): unlike the single-right-hand-side operator,
// whose spin pairs are exchanged by the off-diagonal projectors, no lane ever
// has to move.  Link and clover entries enter as broadcast pairs.
//
// Grid: (site block x pair of right-hand sides) with the pair fastest, so
// that consecutive blocks read the same links and clover (from L2); the
// reducing epilogues stride over the lattice with a grid of resident blocks.
// Consecutive threads take consecutive sites, so every load of a warp is one
// contiguous segment of a field plane.  An odd last pair computes its
// second lane from the first right-hand side and discards it.  A right-hand
// side whose solve has stopped is skipped: nothing of it is stored or
// reduced.
#include <atomic>

#include "device.cuh"
#include "lib.h"
#include "pair.cuh"

namespace qdd {

namespace {

// One complex spinor component of the two right-hand sides: real parts
// (ra, rb) and imaginary parts (ra, rb).
struct CP {
    f2 r, i;
};

// a + k z (rot = false) or a + k i z (rot = true), k a pair of coefficients
template <bool ROT>
__device__ __forceinline__ CP cp_axpy(CP a, f2 k, CP z)
{
    if constexpr (ROT) {
        a.r = pfma(pneg(k), z.i, a.r);
        a.i = pfma(k, z.r, a.i);
    } else {
        a.r = pfma(k, z.r, a.r);
        a.i = pfma(k, z.i, a.i);
    }
    return a;
}

// The 12 components of the FP16 spinors of two right-hand sides at site i.
__device__ __forceinline__ f2 load_pair16(const SpinorView &fa, const SpinorView &fb, unsigned v, unsigned i,
                                          CP (&z)[12])
{
    unsigned wa[12], wb[12];
    const float na = load_words16(fa, v, i, wa);
    const float nb = load_words16(fb, v, i, wb);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        z[k].r = make_float2(hre(wa[k]), hre(wb[k]));
        z[k].i = make_float2(him(wa[k]), him(wb[k]));
    }
    return make_float2(na, nb);
}

// acc += (1 + s gamma_mu) (x) M psi on both right-hand sides, with M = U
// (forward, s = -1) or U^dag (backward, s = +1) and the per-lane coefficient c.
// h_j = u_j + s (X_mu d)_j ; w = M h ; upper += c w ; lower += c s X_mu^dag w.
template <int MU, bool FWD>
__device__ __forceinline__ void hop_rhs2(const CP (&z)[12], const C<float> (&U)[9], f2 c, CP (&acc)[12])
{
    constexpr float s = FWD ? -1.f : 1.f;
    // (X d)_0 and (X d)_1: which lower spin, the sign and whether a factor i
    // enters (x: i d1, i d0; y: -d1, d0; z: i d0, -i d1; t: d0, d1)
    constexpr int p0 = (MU <= 1) ? 1 : 0, p1 = 1 - p0;
    constexpr float k0 = (MU == 1) ? -s : s, k1 = (MU == 2) ? -s : s;
    constexpr bool rot = (MU == 0 || MU == 2);
    CP h[2][3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        h[0][a] = cp_axpy<rot>(z[a], bc2(k0), z[6 + 3 * p0 + a]);
        h[1][a] = cp_axpy<rot>(z[3 + a], bc2(k1), z[6 + 3 * p1 + a]);
    }
    // (X^dag w)_0 and (X^dag w)_1 (x: -i w1, -i w0; y: w1, -w0; z: -i w0, i w1; t: w0, w1),
    // times c s
    constexpr float l0 = (MU == 0 || MU == 2) ? -s : s, l1 = (MU == 0 || MU == 1) ? -s : s;
    const f2 cl0 = make_float2(l0 * c.x, l0 * c.y), cl1 = make_float2(l1 * c.x, l1 * c.y);
#pragma unroll
    for (int sp = 0; sp < 2; sp++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            CP w;
#pragma unroll
            for (int b = 0; b < 3; b++) {
                const C<float> m = FWD ? U[3 * a + b] : C<float>{U[3 * b + a].r, -U[3 * b + a].i};
                if (b == 0) {
                    w.r = pmul(bc2(m.r), h[sp][0].r);
                    w.i = pmul(bc2(m.r), h[sp][0].i);
                } else {
                    w.r = pfma(bc2(m.r), h[sp][b].r, w.r);
                    w.i = pfma(bc2(m.r), h[sp][b].i, w.i);
                }
                w.r = pfma(bc2(-m.i), h[sp][b].i, w.r);
                w.i = pfma(bc2(m.i), h[sp][b].r, w.i);
            }
            // upper spin sp
            acc[3 * sp + a] = cp_axpy<false>(acc[3 * sp + a], c, w);
            // the lower spin q that X^dag w places w_sp in (x, y exchange the spins)
            const int q = (MU <= 1) ? 1 - sp : sp;
            if (q == 0) acc[6 + a] = cp_axpy<rot>(acc[6 + a], cl0, w);
            else acc[9 + a] = cp_axpy<rot>(acc[9 + a], cl1, w);
        }
}

// Both hops in direction MU.
template <int MU>
__device__ __forceinline__ void hop_dir_rhs2(const Geom &g, const SpinorView &ia, const SpinorView &ib,
                                             const LinkView &Ul, unsigned x, const int c[4], float mk, CP (&acc)[12])
{
    const unsigned v = (unsigned)g.V;
    {
        const unsigned xf = (unsigned)fwd_site(g, x, c, MU);
        const float sf = (c[MU] == g.L[MU] - 1 && g.bc[MU] < 0) ? -mk : mk;
        CP z[12];
        C<float> U[9];
        const f2 n = load_pair16(ia, ib, v, xf, z);
        load_link16(Ul, v, MU, x, U);
        hop_rhs2<MU, true>(z, U, make_float2(sf * n.x, sf * n.y), acc);
    }
    {
        const unsigned xb = (unsigned)bwd_site(g, x, c, MU);
        const float sb = (c[MU] == 0 && g.bc[MU] < 0) ? -mk : mk;
        CP z[12];
        C<float> U[9];
        const f2 n = load_pair16(ia, ib, v, xb, z);
        load_link16(Ul, v, MU, xb, U);
        hop_rhs2<MU, false>(z, U, make_float2(sb * n.x, sb * n.y), acc);
    }
}

// acc = sc A psi for both right-hand sides (sc per lane: clover norm times
// spinor norm); the clover entries are decoded once and streamed in storage
// order, each off-diagonal entry applied to both rows it belongs to.
__device__ __forceinline__ void clover_rhs2(const CloverView &A, unsigned v, unsigned i, const CP (&z)[12], f2 sc,
                                            CP (&acc)[12])
{
    const uint4 *p = (const uint4 *)A.d;
    float e[72];   // entry m of block 0 at m, of block 1 at 36 + m (the live ones are kept)
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const uint4 q = p[k * v + i];
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            e[4 * k + j] = hre(w[j]);
            e[36 + 4 * k + j] = him(w[j]);
        }
    }
#pragma unroll
    for (int hb = 0; hb < 2; hb++) {
        const float *E = e + 36 * hb;
        const CP *Z = z + 6 * hb;
        CP o[6];
#pragma unroll
        for (int r = 0; r < 6; r++) {
            o[r].r = pmul(bc2(E[r]), Z[r].r);
            o[r].i = pmul(bc2(E[r]), Z[r].i);
        }
#pragma unroll
        for (int r = 1; r < 6; r++)
#pragma unroll
            for (int j = 0; j < r; j++) {
                const int off = cl_off(r, j);
                const f2 lr = bc2(E[off]), li = bc2(E[off + 1]), ln = bc2(-E[off + 1]);
                o[r].r = pfma(lr, Z[j].r, o[r].r);
                o[r].r = pfma(ln, Z[j].i, o[r].r);
                o[r].i = pfma(lr, Z[j].i, o[r].i);
                o[r].i = pfma(li, Z[j].r, o[r].i);
                o[j].r = pfma(lr, Z[r].r, o[j].r);
                o[j].r = pfma(li, Z[r].i, o[j].r);
                o[j].i = pfma(lr, Z[r].i, o[j].i);
                o[j].i = pfma(ln, Z[r].r, o[j].i);
            }
#pragma unroll
        for (int r = 0; r < 6; r++) {
            acc[6 * hb + r].r = pmul(sc, o[r].r);
            acc[6 * hb + r].i = pmul(sc, o[r].i);
        }
    }
}

// Stores lane L (0: ra, 1: rb) of the pair spinor in FP16 with its site norm.
template <int L>
__device__ __forceinline__ void store_lane16(const SpinorView &f, unsigned v, unsigned i, const CP (&z)[12])
{
    auto lane = [](f2 p) { return L == 0 ? p.x : p.y; };
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(lane(z[k].r)), fabsf(lane(z[k].i))));
    if (!(m >= 1e-30f)) m = 0.f;   // as store_spinor<P16>: tiny sites are stored as zero
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4 *p = (uint4 *)f.d;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        unsigned w[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            __half2 h = __floats2half2_rn(lane(z[4 * q + j].r) * inv, lane(z[4 * q + j].i) * inv);
            w[j] = *reinterpret_cast<unsigned *>(&h);
        }
        p[q * v + i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    f.n[i] = m;
}

// Updates the solver scalars of one right-hand side from its reduced
// epilogue sums (thread 0 of the last block).
template <int EPI>
__device__ __forceinline__ void epi_finish(Scalars *sc, const double (&red)[3], int aux_slot)
{
    if constexpr (EPI == EPI_XMY_NORM) {
        sc->aux[aux_slot] = red[0];
    } else if constexpr (EPI == EPI_RV) {
        const double2 rv = make_double2(red[0], red[1]);
        const double mag2 = rv.x * rv.x + rv.y * rv.y;
        if (!isfinite(mag2) || !isfinite(red[2])) sc->status = S_NONFINITE;
        else if (mag2 <= 1e-60 * sc->rhat2 * red[2]) sc->status = S_BREAK_RV;
        else sc->alpha = zdiv(sc->rho, rv);
    } else if constexpr (EPI == EPI_TS) {
        const double tt = red[2];
        if (!isfinite(tt) || !isfinite(red[0]) || !isfinite(red[1])) sc->status = S_NONFINITE;
        else if (tt == 0.0) sc->status = S_BREAK_TT;
        else sc->omega = make_double2(red[0] / tt, red[1] / tt);
    }
}

constexpr int MR_NT = 256;

template <int EPI>
__global__ void __launch_bounds__(MR_NT, 2) dslash_mrhs_f16_kernel(DslashArgs a)
{
    constexpr int NRED = (EPI == EPI_XMY_NORM) ? 1 : (EPI == EPI_RV || EPI == EPI_TS) ? 3 : 0;
    const long long V = a.g.V;
    const unsigned v = (unsigned)V;
    // pair of right-hand sides fastest: consecutive blocks work on the same
    // sites and share their links and clover through L2
    const unsigned pairs = (unsigned)(a.nrhs + 1) / 2;
    const unsigned pr = blockIdx.x % pairs, sb = blockIdx.x / pairs, nsb = gridDim.x / pairs;
    const int ra = 2 * (int)pr;
    const bool has_b = ra + 1 < a.nrhs;
    const int rb = has_b ? ra + 1 : ra;
    // a right-hand side whose solve has stopped takes no part (uniform per block)
    bool act_a = true, act_b = has_b;
    if constexpr (EPI == EPI_RV || EPI == EPI_TS) {
        act_a = a.sc[ra].status == S_RUN;
        act_b = has_b && a.sc[rb].status == S_RUN;
    }
    if (!act_a && !act_b) return;
    const SpinorView ia = rhs_view<P16>(a.in, V, ra), ib = rhs_view<P16>(a.in, V, rb);
    const SpinorView oa = rhs_view<P16>(a.out, V, ra), ob = rhs_view<P16>(a.out, V, rb);
    const SpinorView ya = rhs_view<P16>(a.y, V, ra), yb = rhs_view<P16>(a.y, V, rb);
    const float mk = -(float)a.kappa;
    f2 part[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};

    auto site = [&](unsigned x) {
        int c[4];
        site_coords(a.g, x, c);
        CP acc[12];
        {
            CP z[12];
            const f2 n = load_pair16(ia, ib, v, x, z);
            const float na = a.A.n[x];
            clover_rhs2(a.A, v, x, z, make_float2(n.x * na, n.y * na), acc);
        }
        hop_dir_rhs2<0>(a.g, ia, ib, a.U, x, c, mk, acc);
        hop_dir_rhs2<1>(a.g, ia, ib, a.U, x, c, mk, acc);
        hop_dir_rhs2<2>(a.g, ia, ib, a.U, x, c, mk, acc);
        hop_dir_rhs2<3>(a.g, ia, ib, a.U, x, c, mk, acc);
        if constexpr (EPI != EPI_D) {
            CP y[12];
            const f2 n = load_pair16(ya, yb, v, x, y);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                y[k].r = pmul(n, y[k].r);
                y[k].i = pmul(n, y[k].i);
            }
            if constexpr (EPI == EPI_XMY || EPI == EPI_XMY_NORM) {
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    acc[k].r = pfma(make_float2(-1.f, -1.f), acc[k].r, y[k].r);
                    acc[k].i = pfma(make_float2(-1.f, -1.f), acc[k].i, y[k].i);
                }
            }
            if constexpr (EPI == EPI_XMY_NORM) {
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    part[0] = pfma(acc[k].r, acc[k].r, part[0]);
                    part[0] = pfma(acc[k].i, acc[k].i, part[0]);
                }
            } else if constexpr (EPI == EPI_RV || EPI == EPI_TS) {
                // RV: <y, out> = sum conj(y) out ; TS: <out, y> = sum conj(out) y
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    const CP &p = EPI == EPI_RV ? y[k] : acc[k];
                    const CP &q = EPI == EPI_RV ? acc[k] : y[k];
                    part[0] = pfma(p.r, q.r, part[0]);
                    part[0] = pfma(p.i, q.i, part[0]);
                    part[1] = pfma(p.r, q.i, part[1]);
                    part[1] = pfma(pneg(p.i), q.r, part[1]);
                    part[2] = pfma(acc[k].r, acc[k].r, part[2]);
                    part[2] = pfma(acc[k].i, acc[k].i, part[2]);
                }
            }
        }
        if (act_a) store_lane16<0>(oa, v, x, acc);
        if (act_b) store_lane16<1>(ob, v, x, acc);
    };

    if constexpr (NRED > 0) {
        for (long long x = (long long)sb * MR_NT + threadIdx.x; x < V; x += (long long)nsb * MR_NT)
            site((unsigned)x);
        // one grid reduction per active right-hand side (each with its own
        // partial sums and arrival counter)
#pragma unroll
        for (int l = 0; l < 2; l++) {
            const bool act = l == 0 ? act_a : act_b;
            if (!act) continue;   // uniform over the block
            const int r = l == 0 ? ra : rb;
            float pl[NRED];
            double red[NRED];
#pragma unroll
            for (int k = 0; k < NRED; k++) pl[k] = l == 0 ? part[k].x : part[k].y;
            if (grid_sum<NRED, float>(pl, red, rs_partials(a.rs, r), rs_counter(a.rs, r), sb, nsb)) {
                double r3[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int k = 0; k < NRED; k++) r3[k] = red[k];
                epi_finish<EPI>(a.sc + r, r3, a.aux_slot);
            }
        }
    } else {
        const long long x = (long long)sb * MR_NT + threadIdx.x;
        if (x < V) site((unsigned)x);
    }
}

template <int EPI>
static long long mrhs_resident(void (*kernel)(DslashArgs))
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, MR_NT, 0) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        v = sms * (per > 0 ? per : 1);
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <int EPI>
static cudaError_t launch_mrhs_epi(const DslashArgs &a, cudaStream_t st)
{
    constexpr bool RED = EPI == EPI_XMY_NORM || EPI == EPI_RV || EPI == EPI_TS;
    void (*kernel)(DslashArgs) = dslash_mrhs_f16_kernel<EPI>;
    const unsigned pairs = (unsigned)(a.nrhs + 1) / 2;
    long long nb = (a.g.V + MR_NT - 1) / MR_NT;
    if constexpr (RED) {
        // a resident grid over all pairs: each block strides over the lattice
        const long long cap = mrhs_resident<EPI>(kernel);
        const long long per_pair = cap > 0 ? (cap + pairs - 1) / pairs : nb;
        if (nb > per_pair) nb = per_pair;
        if (nb > a.rs.max_blocks) nb = a.rs.max_blocks;
    }
    kernel<<<(unsigned)(nb * pairs), MR_NT, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dslash_mrhs_f16(int epi, const DslashArgs &a, cudaStream_t st)
{
    if (a.g.V <= 0) return cudaSuccess;
    if (a.nrhs < 2) return cudaErrorInvalidValue;
    switch (epi) {
    case EPI_D: return launch_mrhs_epi<EPI_D>(a, st);
    case EPI_XMY: return launch_mrhs_epi<EPI_XMY>(a, st);
    case EPI_XMY_NORM: return launch_mrhs_epi<EPI_XMY_NORM>(a, st);
    case EPI_RV: return launch_mrhs_epi<EPI_RV>(a, st);
    case EPI_TS: return launch_mrhs_epi<EPI_TS>(a, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace qdd
