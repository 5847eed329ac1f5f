// ras.cu -- one sweep of the restricted additive Schwarz iteration (Alg. 1
// lines 3-8, Sec. 2) over every domain of the lattice in one launch.
//
// For each domain i (one CTA): the residual is projected onto the extended
// domain Omega'_i (line 4), D_{Omega'_i} v = r is solved approximately with
// the Dirichlet boundary (line 5) by n_dominv minimal-residual iterations
// from zero,
//     q = D rho,  alpha = <q, rho> / <q, q>,  v += alpha rho,  rho -= alpha q,
// and v is restricted to the bulk block Omega_i (line 6) and written there;
// bulk blocks tile the lattice, so the writes of all CTAs form the sum of
// line 8.  Domains are independent (the paper runs one per GPU; here one per
// CTA), so a sweep needs no grid-wide synchronisation.
//
// The Dirichlet operator keeps the clover term on every site of Omega'_i and
// drops every hop whose target lies outside Omega'_i; a direction in which
// the block spans the whole lattice is not decomposed and its hops wrap
// around inside the domain with the boundary sign.  The domain arithmetic is
// FP32 whatever the storage precision of the fields.
//
// Two kernels:
//  * ras_smem_kernel: extended domains of at most RAS_SMEM_MAX_SITES sites.
//    One thread per site; the MR residual rho lives in shared memory (read
//    by the neighbours' hops), q and v in registers; links and clover come
//    through L1.
//  * ras_gmem_kernel: any domain size.  A persistent grid of `slots` CTAs
//    loops over the domains; rho, q and v of the current domain live in a
//    per-CTA slot of global scratch (L2-resident for moderate domains).
//  * ras_cluster_kernel: 6^4 or 8^4 extended domains (overlap on 4^4 blocks),
//    one thread-block cluster per domain.
//  * the phased sweep (ras_phase_*): few large domains, each spread over many
//    CTAs, one launch per MR step.
//
// The same kernels run the other members of the Schwarz family: a sweep of
// the multiplicative SAP solves only the domains of one colour of the
// red/black block ordering (the others write zero), and a sweep of plain
// additive Schwarz adds each domain's solution on all its extended sites into
// an FP32 sum (atomic additions: the extended domains overlap), which
// as_finish_kernel then writes out.
#include <atomic>
#include <cstring>

#include "device.cuh"
#include "lib.h"
#include "pair.cuh"
#include "tma.cuh"
#include "tmem.cuh"

namespace qdd {

struct DomSite {
    long long x;      // global site
    bool act, bulk;
    int nf[4], nb[4]; // local neighbour index, -1 when the hop leaves the domain
    long long xb[4];  // global backward neighbour (its link is U_mu(x - mu))
    float cf[4], cb[4];
};

// n / d for 0 <= n < 2^31 with the divisor's precomputed multiplier
__device__ __forceinline__ int fast_div(int n, int d, unsigned m, int sh)
{
    return d >= 2 ? (int)(__umulhi((unsigned)n, m) >> sh) : n;
}

__device__ __forceinline__ void dom_site(const Geom &g, const DomainGeom &dg, int dom, int l, float kappa,
                                         DomSite &s)
{
    s.act = l < dg.nloc;
    const int ll = s.act ? l : 0;
    int k[4], lc[4], gc[4];
    {
        int r = dom;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            const int q = fast_div(r, dg.nb[mu], dg.nb_m[mu], dg.nb_sh[mu]);
            k[mu] = r - q * dg.nb[mu];
            r = q;
        }
        r = ll;
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            const int q = fast_div(r, dg.e[mu], dg.e_m[mu], dg.e_sh[mu]);
            lc[mu] = r - q * dg.e[mu];
            r = q;
        }
    }
    s.x = 0;
    s.bulk = s.act;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        int v = k[mu] * dg.b[mu] - dg.sh[mu] + lc[mu];  // in (-L, 2L)
        if (v < 0) v += g.L[mu];
        else if (v >= g.L[mu]) v -= g.L[mu];
        gc[mu] = v;
        s.x += (long long)v * g.stride[mu];
        if (lc[mu] < dg.sh[mu] || lc[mu] >= dg.sh[mu] + dg.b[mu]) s.bulk = false;
    }
    int lstride = 1;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int e = dg.e[mu];
        const bool whole = dg.b[mu] == g.L[mu];
        if (whole) {
            s.nf[mu] = lc[mu] == e - 1 ? ll - (e - 1) * lstride : ll + lstride;
            s.nb[mu] = lc[mu] == 0 ? ll + (e - 1) * lstride : ll - lstride;
        } else {
            s.nf[mu] = lc[mu] + 1 < e ? ll + lstride : -1;
            s.nb[mu] = lc[mu] > 0 ? ll - lstride : -1;
        }
        s.cf[mu] = (gc[mu] == g.L[mu] - 1 && g.bc[mu] < 0) ? kappa : -kappa;
        s.cb[mu] = (gc[mu] == 0 && g.bc[mu] < 0) ? kappa : -kappa;
        s.xb[mu] = bwd_site(g, s.x, gc, mu);
        lstride *= e;
    }
}

// Local spinor from a planar float2 [12][stride] array (shared or global).
// Domain-local FP32 spinors: 6 planes of float4 (two complex each), so that
// a spinor moves in 6 wide accesses.  base must be 16-byte aligned; the
// buffers are declared as float2 [12][stride], the same footprint.
__device__ __forceinline__ void ld_local(const float2 *base, int stride, int l, C<float> (&s)[12])
{
    const float4 *b = reinterpret_cast<const float4 *>(base);
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const float4 v = b[q * stride + l];
        s[2 * q] = {v.x, v.y};
        s[2 * q + 1] = {v.z, v.w};
    }
}

__device__ __forceinline__ void st_local(float2 *base, int stride, int l, const C<float> (&s)[12])
{
    float4 *b = reinterpret_cast<float4 *>(base);
#pragma unroll
    for (int q = 0; q < 6; q++) b[q * stride + l] = make_float4(s[2 * q].r, s[2 * q].i, s[2 * q + 1].r, s[2 * q + 1].i);
}

// The split spin-pair layout of the packed domain solve (ras_mr_domain_x2):
// float4 [6][stride], group g = 3 h + a (h = 0: spins 0, 1; h = 1: spins 2, 3;
// a the colour) holds (psi[2h][a].re, psi[2h+1][a].re, psi[2h][a].im,
// psi[2h+1][a].im), i.e. the real-part pair and the imaginary-part pair of
// the two spins.  Same footprint as ld_local / st_local.
__device__ __forceinline__ void st_split(float2 *base, int stride, int l, const C<float> (&s)[12])
{
    float4 *b = reinterpret_cast<float4 *>(base);
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int a = 0; a < 3; a++)
            b[(3 * h + a) * stride + l] =
                make_float4(s[6 * h + a].r, s[6 * h + 3 + a].r, s[6 * h + a].i, s[6 * h + 3 + a].i);
}

__device__ __forceinline__ void ld_split(const float2 *base, int stride, int l, C<float> (&s)[12])
{
    const float4 *b = reinterpret_cast<const float4 *>(base);
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float4 v = b[(3 * h + a) * stride + l];
            s[6 * h + a] = {v.x, v.z};
            s[6 * h + 3 + a] = {v.y, v.w};
        }
}

template <int P, int MU>
__device__ __forceinline__ void dom_hops(const RasArgs &a, const DomSite &ds, const float2 *rho, int stride,
                                         C<float> (&q)[12])
{
    const long long V = a.g.V;
    if (ds.nf[MU] >= 0) {
        C<float> s[12], U[9];
        ld_local(rho, stride, ds.nf[MU], s);
        load_link<P>(a.U, V, MU, ds.x, U);
        hop<MU, true>(q, s, U, ds.cf[MU]);
    }
    if (ds.nb[MU] >= 0) {
        C<float> s[12], U[9];
        ld_local(rho, stride, ds.nb[MU], s);
        load_link<P>(a.U, V, MU, ds.xb[MU], U);
        hop<MU, false>(q, s, U, ds.cb[MU]);
    }
}

// q = D_{Omega'} rho at one local site.
template <int P>
__device__ __forceinline__ void dom_apply(const RasArgs &a, const DomSite &ds, const C<float> (&own)[12],
                                          const float2 *rho, int stride, C<float> (&q)[12])
{
    float av[72];
    load_clover<P>(a.A, a.g.V, ds.x, av);
    clover_apply(av, own, q);
    dom_hops<P, 0>(a, ds, rho, stride, q);
    dom_hops<P, 1>(a, ds, rho, stride, q);
    dom_hops<P, 2>(a, ds, rho, stride, q);
    dom_hops<P, 3>(a, ds, rho, stride, q);
}

template <int P>
__device__ __forceinline__ void write_outputs_to(SpinorView vout, SpinorView acc, int accumulate, long long V,
                                                 long long x, const C<float> (&v)[12])
{
    typedef typename RealOf<P>::T T;
    if (vout.d) store_spinor<P>(vout, V, x, v);
    if (accumulate) {
        C<T> o[12];
        load_spinor<P>(acc, V, x, o);
#pragma unroll
        for (int k = 0; k < 12; k++) o[k] = cadd(o[k], C<T>{(T)v[k].r, (T)v[k].i});
        store_spinor<P>(acc, V, x, o);
    } else {
        store_spinor<P>(acc, V, x, v);
    }
}

template <int P>
__device__ __forceinline__ void write_outputs(const RasArgs &a, long long x, const C<float> (&v)[12])
{
    write_outputs_to<P>(a.vout, a.acc, a.accumulate, a.g.V, x, v);
}

// Bulk site of a domain that this SAP sweep does not solve: v = 0 there.
template <int P>
__device__ __forceinline__ void zero_outputs(const RasArgs &a, long long x)
{
    C<float> z[12];
#pragma unroll
    for (int k = 0; k < 12; k++) z[k] = {0.f, 0.f};
    if (a.vout.d) store_spinor<P>(a.vout, a.g.V, x, z);
    if (!a.accumulate) store_spinor<P>(a.acc, a.g.V, x, z);
}

// Additive Schwarz: the domain's solution at one of its extended sites,
// added to the sum of all domains covering that site (asum already offset to
// this right-hand side; complex pair k of the site in float4 plane k).
__device__ __forceinline__ void as_add(const RasArgs &a, long long x, const C<float> (&v)[12])
{
#pragma unroll
    for (int k = 0; k < 6; k++)
        atomicAdd(&a.asum[(long long)k * a.g.V + x],
                  make_float4(v[2 * k].r, v[2 * k].i, v[2 * k + 1].r, v[2 * k + 1].i));
}

// Colour of a domain in the red/black block ordering: parity of the sum of
// its block coordinates.
__device__ __forceinline__ int dom_color(const DomainGeom &dg, int dom)
{
    int sum = 0, r = dom;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int q = fast_div(r, dg.nb[mu], dg.nb_m[mu], dg.nb_sh[mu]);
        sum += r - q * dg.nb[mu];
        r = q;
    }
    return sum & 1;
}

__device__ __forceinline__ bool skip_domain(const RasArgs &a, int dom)
{
    return a.color != 0 && dom_color(a.dg, dom) != a.color - 1;
}

// The sweep's input at site x: `in`, or with a fused BiCGStab update
// r + b y + c v (y = in for RAS_FUSE_P, absent for RAS_FUSE_S) in FP32.
template <int P>
__device__ __forceinline__ void staged_input(const RasArgs &a, long long V, long long x, C<float> b, C<float> c,
                                             C<float> (&out)[12])
{
    if (a.fuse == RAS_FUSE_NONE) {
        load_spinor<P>(a.in, V, x, out);
        return;
    }
    C<float> t[12];
    load_spinor<P>(a.fr, V, x, out);
    load_spinor<P>(a.fz, V, x, t);
#pragma unroll
    for (int k = 0; k < 12; k++) out[k] = cfma(c, t[k], out[k]);
    if (a.fuse == RAS_FUSE_P) {
        load_spinor<P>(a.in, V, x, t);
#pragma unroll
        for (int k = 0; k < 12; k++) out[k] = cfma(b, t[k], out[k]);
    }
}

// Coefficients (b, c) of the fused update from the solver scalars.
__device__ __forceinline__ void fuse_coefs(const RasArgs &a, int rr, C<float> &b, C<float> &c)
{
    b = {0.f, 0.f};
    c = {0.f, 0.f};
    if (a.fuse == RAS_FUSE_P) {
        const double2 be = a.sc[rr].beta, om = a.sc[rr].omega;
        b = {(float)be.x, (float)be.y};
        const double2 bo = zmul(be, om);
        c = {(float)-bo.x, (float)-bo.y};
    } else if (a.fuse == RAS_FUSE_S) {
        const double2 al = a.sc[rr].alpha;
        c = {(float)-al.x, (float)-al.y};
    }
}

// Compact description of one site of the extended domain held by a thread
// of the shared-memory kernel.
struct LocSite {
    int x;           // global site index
    unsigned m;      // bit mu / 4+mu: forward / backward hop kept (inside the domain)
                     // bit 8+mu / 12+mu: that hop carries the boundary sign -1
                     // bit 16+mu / 20+mu: that hop wraps around a whole-lattice direction
    int ls[4];       // local strides
    int e[4];
};

enum { M_ACT = 1u << 24, M_BULK = 1u << 25 };

__device__ __forceinline__ void loc_site(const Geom &g, const DomainGeom &dg, int dom, int l, LocSite &s)
{
    int k[4], lc[4];
    int r = dom;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int q = fast_div(r, dg.nb[mu], dg.nb_m[mu], dg.nb_sh[mu]);
        k[mu] = r - q * dg.nb[mu];
        r = q;
    }
    const bool act = l < dg.nloc;
    r = act ? l : 0;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int q = fast_div(r, dg.e[mu], dg.e_m[mu], dg.e_sh[mu]);
        lc[mu] = r - q * dg.e[mu];
        r = q;
    }
    unsigned m = act ? (unsigned)M_ACT : 0u;
    bool bulk = act;
    long long x = 0;
    int ls = 1;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        // k b - sh + lc lies in (-L, 2L): one conditional wrap
        int gc = k[mu] * dg.b[mu] - dg.sh[mu] + lc[mu];
        if (gc < 0) gc += g.L[mu];
        else if (gc >= g.L[mu]) gc -= g.L[mu];
        x += (long long)gc * g.stride[mu];
        if (lc[mu] < dg.sh[mu] || lc[mu] >= dg.sh[mu] + dg.b[mu]) bulk = false;
        const int e = dg.e[mu];
        const bool whole = dg.b[mu] == g.L[mu];
        if (whole || lc[mu] + 1 < e) m |= 1u << mu;
        if (whole || lc[mu] > 0) m |= 1u << (4 + mu);
        if (whole && lc[mu] == e - 1) m |= 1u << (16 + mu);
        if (whole && lc[mu] == 0) m |= 1u << (20 + mu);
        if (g.bc[mu] < 0 && gc == g.L[mu] - 1) m |= 1u << (8 + mu);
        if (g.bc[mu] < 0 && gc == 0) m |= 1u << (12 + mu);
        s.ls[mu] = ls;
        s.e[mu] = e;
        ls *= e;
    }
    if (bulk) m |= M_BULK;
    s.m = m;
    s.x = (int)x;
}

// Shared-memory layout of one CTA (one domain, NT threads):
//   rho  float4[6][NT]    MR residual (read by the neighbours' hops)
//   v    float4[6][NT]    MR solution
//   U    links of the domain's sites, 4 directions, in the storage format of
//        the field (FP16: uint2[12][NT], FP32: float4[12][NT]); the backward hop
//        from a site uses the forward link of its neighbour, which is inside
//        the domain whenever the hop is kept
//   A    clover (only when SC): FP16 uint4[9][NT] + float[NT], FP32 float4[18][NT]
//
// Expanded variant (EXP): links are staged as full 18-real FP32 matrices
// (float2[4][9][NT], third row rebuilt once) and the clover as FP32
// (float4[18][NT], FP16 norm applied once), so that the MR iterations do no
// conversions and no row rebuilds: 768 B per site, for small domains.
template <int P, bool EXP> struct RasSmem {
    static constexpr size_t link_bytes = EXP ? 288 : (P == P16 ? 96 : 192);
    static constexpr size_t clover_bytes = EXP ? 288 : (P == P16 ? 148 : 288);
    static constexpr size_t clover_data = EXP ? 288 : (P == P16 ? 144 : 288);
    static constexpr size_t bytes(int nt, bool sc) { return (size_t)nt * (192 + link_bytes + (sc ? clover_bytes : 0)); }
};

template <int P, bool EXP>
__device__ __forceinline__ void smem_link(LinkView sU, int NT, int mu, int l, C<float> (&U)[9])
{
    if constexpr (EXP) {
        const float2 *p = (const float2 *)sU.d + mu * 9 * NT;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const float2 v = p[k * NT + l];
            U[k] = {v.x, v.y};
        }
    } else {
        load_link<P>(sU, NT, mu, l, U);
    }
}

template <int P, bool EXP, int MU>
__device__ __forceinline__ void smem_hops(const LocSite &s, int l, const float2 *srho, LinkView sU, float kappa,
                                          C<float> (&q)[12], int NT)
{
    const int ls = s.ls[MU], e = s.e[MU];
    if (s.m & (1u << MU)) {
        const int nf = (s.m & (1u << (16 + MU))) ? l - (e - 1) * ls : l + ls;
        C<float> n[12], U[9];
        ld_local(srho, NT, nf, n);
        smem_link<P, EXP>(sU, NT, MU, l, U);
        hop<MU, true>(q, n, U, (s.m & (1u << (8 + MU))) ? kappa : -kappa);
    }
    if (s.m & (1u << (4 + MU))) {
        const int nb = (s.m & (1u << (20 + MU))) ? l + (e - 1) * ls : l - ls;
        C<float> n[12], U[9];
        ld_local(srho, NT, nb, n);
        smem_link<P, EXP>(sU, NT, MU, nb, U);
        hop<MU, false>(q, n, U, (s.m & (1u << (12 + MU))) ? kappa : -kappa);
    }
}

// The N_dominv minimal-residual iterations of one domain on its staged
// residual (srho, FP32), with v (sv) starting at zero, and the restriction of
// v to the bulk sites.  All NT threads of the CTA call it.
template <int P, int NT, bool SC, bool EXP>
__device__ __forceinline__ void ras_mr_domain(const RasArgs &a, const LocSite &s, float2 *srho, float2 *sv,
                                              unsigned char *sA, const LinkView &lU, const CloverView &lA,
                                              float (&wpart)[3][NT / 32]);

template <int NT, bool TM = false>
__device__ __forceinline__ void ras_mr_domain_x2(const RasArgs &a, const LocSite &s, float2 *srho, float2 *sv,
                                                 const unsigned char *sA, const float *sAn, const LinkView &lU,
                                                 float (&wpart)[3][NT / 32], unsigned tv = 0);

template <int P, int NT, bool SC, bool EXP>
__device__ __forceinline__ void ras_mr_domain(const RasArgs &a, const LocSite &s, float2 *srho, float2 *sv,
                                              unsigned char *sA, const LinkView &lU, const CloverView &lA,
                                              float (&wpart)[3][NT / 32])
{
    if constexpr (P == P16 && SC && !EXP) {
        ras_mr_domain_x2<NT>(a, s, srho, sv, sA, lA.n, lU, wpart);
        return;
    }
    const long long V = a.g.V;
    const int l = threadIdx.x;
    const bool act = s.m & M_ACT;
    for (int it = 0; it < a.n_iter; it++) {
        __syncthreads();
        C<float> q[12];
#pragma unroll
        for (int k = 0; k < 12; k++) q[k] = {0.f, 0.f};
        if (act) {
            {
                C<float> own[12];
                float av[72];
                ld_local(srho, NT, l, own);
                if constexpr (EXP) {
                    load_clover<P32>(CloverView{sA, nullptr}, NT, l, av);
                    clover_apply(av, own, q);
                } else {
                    const float na = load_clover_u<P>(lA, SC ? (long long)NT : V, SC ? l : s.x, av);
                    clover_apply(av, own, q);
                    if constexpr (P == P16) {
#pragma unroll
                        for (int k = 0; k < 12; k++) q[k] = cscale(q[k], na);
                    }
                }
            }
            smem_hops<P, EXP, 0>(s, l, srho, lU, a.kappa, q, NT);
            smem_hops<P, EXP, 1>(s, l, srho, lU, a.kappa, q, NT);
            smem_hops<P, EXP, 2>(s, l, srho, lU, a.kappa, q, NT);
            smem_hops<P, EXP, 3>(s, l, srho, lU, a.kappa, q, NT);
        }
        // <q, rho> and |q|^2 over the domain in FP32: warp sums, then every
        // thread adds the per-warp partials itself (one barrier; the next write
        // of wpart comes after the next iteration's first barrier)
        float red[3];
        {
            C<float> own[12];
            ld_local(srho, NT, l, own);
            float qr = 0.f, qi = 0.f, qq = 0.f;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                cdot_acc(q[k], own[k], qr, qi);
                cnorm_acc(q[k], qq);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                qr += __shfl_xor_sync(0xffffffffu, qr, o);
                qi += __shfl_xor_sync(0xffffffffu, qi, o);
                qq += __shfl_xor_sync(0xffffffffu, qq, o);
            }
            if ((l & 31) == 0) {
                wpart[0][l >> 5] = qr;
                wpart[1][l >> 5] = qi;
                wpart[2][l >> 5] = qq;
            }
            __syncthreads();
            red[0] = red[1] = red[2] = 0.f;
#pragma unroll
            for (int w = 0; w < NT / 32; w++) {
                red[0] += wpart[0][w];
                red[1] += wpart[1][w];
                red[2] += wpart[2][w];
            }
        }
        // every thread is past the barrier above: all reads of rho for this
        // iteration are done and rho can be updated in place
        if (red[2] > 0.f) {
            const float inv = 1.0f / red[2];
            const C<float> al = {red[0] * inv, red[1] * inv};
            C<float> own[12], vv[12];
            ld_local(srho, NT, l, own);
            ld_local(sv, NT, l, vv);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                vv[k] = cfma(al, own[k], vv[k]);
                own[k] = cfma(cneg(al), q[k], own[k]);
            }
            st_local(sv, NT, l, vv);
            st_local(srho, NT, l, own);
        }
    }
    if (a.asum) {  // additive Schwarz: no restriction, overlaps summed
        if (act) {
            C<float> vv[12];
            ld_local(sv, NT, l, vv);
            as_add(a, s.x, vv);
        }
    } else if (s.m & M_BULK) {  // restriction R_{Omega}
        C<float> vv[12];
        ld_local(sv, NT, l, vv);
        write_outputs<P>(a, s.x, vv);
    }
}

// Whether a sweep kernel runs the packed domain solve (FP16 storage with the
// clover staged in shared memory in its compact form): then rho and v live
// in the split spin-pair layout.
template <int P, bool SC, bool EXP> struct SplitRho {
    static constexpr bool value = P == P16 && SC && !EXP;
};

// Row 2 of the staged FP16 links, rebuilt once per sweep instead of in
// every MR iteration: entry k of link mu of site i at r2[(3 mu + k) v + i]
// (FP32 complex).  Rebuilding it in every hop cost 10% of the sweep.
__device__ __forceinline__ void stage_row2(const LinkView &u, float2 *r2, unsigned v, unsigned i)
{
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        C<float> U[9];
        load_link16(u, v, mu, i, U);
#pragma unroll
        for (int k = 0; k < 3; k++) r2[(3 * mu + k) * v + i] = make_float2(U[6 + k].r, U[6 + k].i);
    }
}

// The staged FP16 link U_mu of site i (rows 0 and 1) with its staged row 2.
__device__ __forceinline__ void load_link16_r2(const LinkView &u, const float2 *r2, unsigned v, int mu, unsigned i,
                                               C<float> (&U)[9])
{
    const uint2 *p = (const uint2 *)u.d + mu * 3 * v;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const uint2 w = p[q * v + i];
        U[2 * q] = {hre(w.x), him(w.x)};
        U[2 * q + 1] = {hre(w.y), him(w.y)};
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float2 w = r2[(3 * mu + k) * v + i];
        U[6 + k] = {w.x, w.y};
    }
}

// Both hops of direction MU on the split residual in shared memory (float4
// groups), links from the staged FP16 planes (row 2 from r2 when R2).
template <int MU, bool R2>
__device__ __forceinline__ void smem_hops_x2(const LocSite &s, int l, const float4 *R4, const LinkView &sU,
                                             const float2 *r2, float kappa, int NT, f2 (&AUR)[3], f2 (&AUI)[3],
                                             f2 (&ADR)[3], f2 (&ADI)[3])
{
    const int ls = s.ls[MU], e = s.e[MU];
    // the neighbour's spin pairs; for MU = 0, 1 the lower spins exchanged
    // (float4 loads: scalar loads at a 16-byte stride would cost four
    // shared-memory wavefronts each)
    auto pairs = [&](int n, f2 (&UR)[3], f2 (&UI)[3], f2 (&DA)[3], f2 (&DB)[3]) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float4 u = R4[a * NT + n];
            const float4 d = R4[(3 + a) * NT + n];
            UR[a] = make_float2(u.x, u.y);
            UI[a] = make_float2(u.z, u.w);
            if constexpr (MU >= 2) {
                DA[a] = make_float2(d.x, d.y);
                DB[a] = make_float2(d.z, d.w);
            } else {
                DA[a] = make_float2(d.y, d.x);
                DB[a] = make_float2(d.w, d.z);
            }
        }
    };
    // dropped hops (Dirichlet boundary) run with coefficient 0 on the site's
    // own data instead of branching around them: a branch around the packed
    // accumulators made the compiler move them at every join
    const bool kf = s.m & (1u << MU), kb = s.m & (1u << (4 + MU));
    if (MU == 3 ? kf : true) {   // t hops: uniform over a warp of these domains, branched
        const int nf = !kf ? l : (s.m & (1u << (16 + MU))) ? l - (e - 1) * ls : l + ls;
        f2 UR[3], UI[3], DA[3], DB[3];
        C<float> U[9];
        pairs(nf, UR, UI, DA, DB);
        if constexpr (R2) load_link16_r2(sU, r2, (unsigned)NT, MU, (unsigned)l, U);
        else load_link16(sU, (unsigned)NT, MU, (unsigned)l, U);
        const float c = !kf ? 0.f : (s.m & (1u << (8 + MU))) ? kappa : -kappa;
        hop_core<MU, true>(UR, UI, DA, DB, U, c, AUR, AUI, ADR, ADI);
    }
    if (MU == 3 ? kb : true) {
        const int nb = !kb ? l : (s.m & (1u << (20 + MU))) ? l + (e - 1) * ls : l - ls;
        f2 UR[3], UI[3], DA[3], DB[3];
        C<float> U[9];
        pairs(nb, UR, UI, DA, DB);
        if constexpr (R2) load_link16_r2(sU, r2, (unsigned)NT, MU, (unsigned)nb, U);
        else load_link16(sU, (unsigned)NT, MU, (unsigned)nb, U);
        const float c = !kb ? 0.f : (s.m & (1u << (12 + MU))) ? kappa : -kappa;
        hop_core<MU, false>(UR, UI, DA, DB, U, c, AUR, AUI, ADR, ADI);
    }
}

// ras_mr_domain on packed FP32 pairs (FFMA2, pair.cuh) for FP16 fields with
// the compact staged clover: rho and v in the split layout (st_split), the
// hops' two spins as pairs.  The same MR
// arithmetic in FP32; only its grouping into instructions differs.
// The clover term stays scalar (see below).  Measured at 32^4 against the
// all-scalar solve: 4x4x4x2 domains, N_dominv 3: 240.5 -> 215.7 us; 4^4
// domains, N_dominv 4: 328 -> 304 us.
//
// With TM (the TMA-staged sweep): v lives in tensor memory at this thread's
// lane (24 columns from tv, the split layout's 6 float4 groups), and sv holds
// the links' row 2 (stage_row2) instead of v.
template <int NT, bool TM>
__device__ __forceinline__ void ras_mr_domain_x2(const RasArgs &a, const LocSite &s, float2 *srho, float2 *sv,
                                                 const unsigned char *sA, const float *sAn, const LinkView &lU,
                                                 float (&wpart)[3][NT / 32], unsigned tv)
{
    const int l = threadIdx.x;
    const bool act = s.m & M_ACT;
    float4 *R4 = reinterpret_cast<float4 *>(srho);
    float4 *V4 = reinterpret_cast<float4 *>(sv);
    for (int it = 0; it < a.n_iter; it++) {
        __syncthreads();
        f2 AUR[3], AUI[3], ADR[3], ADI[3];
#pragma unroll
        for (int c = 0; c < 3; c++) AUR[c] = AUI[c] = ADR[c] = ADI[c] = make_float2(0.f, 0.f);
        if (act) {
            // the clover term in scalar FP32 arithmetic: written on the
            // packed pairs (block 0, block 1) the compiler added about 250
            // register moves per site and iteration, and the solve ran 7%
            // slower
            {
                C<float> own[12], o[12];
                float av[72];
                ld_split(srho, NT, l, own);
                const float na = load_clover_u<P16>(CloverView{sA, sAn}, NT, l, av);
                clover_apply(av, own, o);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    AUR[c] = make_float2(na * o[c].r, na * o[3 + c].r); AUI[c] = make_float2(na * o[c].i, na * o[3 + c].i);
                    ADR[c] = make_float2(na * o[6 + c].r, na * o[9 + c].r); ADI[c] = make_float2(na * o[6 + c].i, na * o[9 + c].i);
                }
            }
            smem_hops_x2<0, TM>(s, l, R4, lU, sv, a.kappa, NT, AUR, AUI, ADR, ADI);
            smem_hops_x2<1, TM>(s, l, R4, lU, sv, a.kappa, NT, AUR, AUI, ADR, ADI);
            smem_hops_x2<2, TM>(s, l, R4, lU, sv, a.kappa, NT, AUR, AUI, ADR, ADI);
            smem_hops_x2<3, TM>(s, l, R4, lU, sv, a.kappa, NT, AUR, AUI, ADR, ADI);
        }
        // <q, rho> = sum conj(q) rho and |q|^2 on pairs, then over the domain
        // in FP32 (warp sums, per-warp partials read by every thread)
        f2 RR[6], RI[6];
        float red[3];
        {
            f2 d0 = make_float2(0.f, 0.f), d1 = d0, d2 = d0;
#pragma unroll
            for (int g = 0; g < 6; g++) {
                const float4 r = R4[g * NT + l];
                RR[g] = make_float2(r.x, r.y);
                RI[g] = make_float2(r.z, r.w);
                const f2 QR = g < 3 ? AUR[g] : ADR[g - 3], QI = g < 3 ? AUI[g] : ADI[g - 3];
                d0 = pfma(QR, RR[g], d0);
                d0 = pfma(QI, RI[g], d0);
                d1 = pfma(QR, RI[g], d1);
                d1 = pfma(pneg(QI), RR[g], d1);
                d2 = pfma(QR, QR, d2);
                d2 = pfma(QI, QI, d2);
            }
            float qr = d0.x + d0.y, qi = d1.x + d1.y, qq = d2.x + d2.y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                qr += __shfl_xor_sync(0xffffffffu, qr, o);
                qi += __shfl_xor_sync(0xffffffffu, qi, o);
                qq += __shfl_xor_sync(0xffffffffu, qq, o);
            }
            if ((l & 31) == 0) {
                wpart[0][l >> 5] = qr;
                wpart[1][l >> 5] = qi;
                wpart[2][l >> 5] = qq;
            }
            __syncthreads();
            red[0] = red[1] = red[2] = 0.f;
#pragma unroll
            for (int w = 0; w < NT / 32; w++) {
                red[0] += wpart[0][w];
                red[1] += wpart[1][w];
                red[2] += wpart[2][w];
            }
        }
        // every thread is past the barrier: rho can be updated in place
        if (red[2] > 0.f) {  // uniform over the CTA (the warp-wide TMEM accesses need that)
            const float inv = 1.0f / red[2];
            const f2 ar = bc2(red[0] * inv), ai = bc2(red[1] * inv), an = bc2(-red[1] * inv);
            float vt[TM ? 24 : 1];
            if constexpr (TM) {
                tm_ld24(tv, vt);
            }
#pragma unroll
            for (int g = 0; g < 6; g++) {
                const f2 QR = g < 3 ? AUR[g] : ADR[g - 3], QI = g < 3 ? AUI[g] : ADI[g - 3];
                f2 VR, VI;
                if constexpr (TM) {
                    VR = make_float2(vt[4 * g], vt[4 * g + 1]);
                    VI = make_float2(vt[4 * g + 2], vt[4 * g + 3]);
                } else {
                    const float4 vq = V4[g * NT + l];
                    VR = make_float2(vq.x, vq.y);
                    VI = make_float2(vq.z, vq.w);
                }
                // v += alpha rho
                VR = pfma(ar, RR[g], VR);
                VR = pfma(an, RI[g], VR);
                VI = pfma(ar, RI[g], VI);
                VI = pfma(ai, RR[g], VI);
                // rho -= alpha q
                f2 NR = pfma(pneg(ar), QR, RR[g]);
                NR = pfma(ai, QI, NR);
                f2 NI = pfma(pneg(ar), QI, RI[g]);
                NI = pfma(an, QR, NI);
                if constexpr (TM) {
                    vt[4 * g] = VR.x;
                    vt[4 * g + 1] = VR.y;
                    vt[4 * g + 2] = VI.x;
                    vt[4 * g + 3] = VI.y;
                } else {
                    V4[g * NT + l] = make_float4(VR.x, VR.y, VI.x, VI.y);
                }
                R4[g * NT + l] = make_float4(NR.x, NR.y, NI.x, NI.y);
            }
            if constexpr (TM) {
                tm_st8(tv, vt);
                tm_st8(tv + 8, vt + 8);
                tm_st8(tv + 16, vt + 16);
            }
        }
    }
    if constexpr (TM) {  // (the TMA-staged sweeps never sum overlaps: no asum)
        float vt[24];
        tm_ld24(tv, vt);  // by every thread: the warp-wide load precedes the branch
        if (s.m & M_BULK) {  // restriction R_{Omega}
            C<float> vv[12];
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const int g = 3 * h + c;
                    vv[6 * h + c] = {vt[4 * g], vt[4 * g + 2]};
                    vv[6 * h + 3 + c] = {vt[4 * g + 1], vt[4 * g + 3]};
                }
            write_outputs<P16>(a, s.x, vv);
        }
    } else if (a.asum) {  // additive Schwarz: no restriction, overlaps summed
        if (act) {
            C<float> vv[12];
            ld_split(sv, NT, l, vv);
            as_add(a, s.x, vv);
        }
    } else if (s.m & M_BULK) {  // restriction R_{Omega}
        C<float> vv[12];
        ld_split(sv, NT, l, vv);
        write_outputs<P16>(a, s.x, vv);
    }
}

template <int P, int NT, bool SC, bool EXP>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) ras_smem_kernel(RasArgs a)
{
    const int rr = blockIdx.x % a.nrhs, dom = blockIdx.x / a.nrhs;
    if (a.sc && a.sc[rr].status != S_RUN) return;
    a.in = rhs_view<P>(a.in, a.g.V, rr);
    a.vout = rhs_view<P>(a.vout, a.g.V, rr);
    a.acc = rhs_view<P>(a.acc, a.g.V, rr);
    a.fr = rhs_view<P>(a.fr, a.g.V, rr);
    a.fz = rhs_view<P>(a.fz, a.g.V, rr);
    if (a.asum) a.asum += (long long)rr * 6 * a.g.V;
    C<float> fb, fc;
    fuse_coefs(a, rr, fb, fc);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float wpart[3][NT / 32];
    float2 *srho = reinterpret_cast<float2 *>(smem);
    float2 *sv = srho + 12 * NT;
    unsigned char *sU = reinterpret_cast<unsigned char *>(sv + 12 * NT);
    unsigned char *sA = sU + (size_t)NT * RasSmem<P, EXP>::link_bytes;
    float *sAn = reinterpret_cast<float *>(sA + (size_t)NT * RasSmem<P, EXP>::clover_data);
    const LinkView lU{sU};
    const CloverView lA = SC ? CloverView{sA, sAn} : a.A;
    const long long V = a.g.V;
    const int l = threadIdx.x;
    LocSite s;
    loc_site(a.g, a.dg, dom, l, s);
    const bool act = s.m & M_ACT;
    if (skip_domain(a, dom)) {  // uniform over the CTA, before any barrier
        if (s.m & M_BULK) zero_outputs<P>(a, s.x);
        return;
    }

    // stage the projection P_{Omega'} r, and the domain's links and clover
    {
        C<float> r[12], z[12];
#pragma unroll
        for (int k = 0; k < 12; k++) { r[k] = {0.f, 0.f}; z[k] = {0.f, 0.f}; }
        if (act) {
            staged_input<P>(a, V, s.x, fb, fc, r);
            // the fused update's result, on the bulk sites (each written once)
            if (a.fuse != RAS_FUSE_NONE && (s.m & M_BULK)) store_spinor<P>(a.in, V, s.x, r);
        }
        if constexpr (SplitRho<P, SC, EXP>::value) {
            st_split(srho, NT, l, r);
            st_split(sv, NT, l, z);
        } else {
            st_local(srho, NT, l, r);
            st_local(sv, NT, l, z);
        }
        if (act) {
            if constexpr (EXP) {
#pragma unroll 1
                for (int mu = 0; mu < 4; mu++) {
                    C<float> U[9];
                    load_link<P>(a.U, V, mu, s.x, U);
#pragma unroll
                    for (int k = 0; k < 9; k++) ((float2 *)sU)[(mu * 9 + k) * NT + l] = make_float2(U[k].r, U[k].i);
                }
                float av[72];
                load_clover<P>(a.A, V, s.x, av);
#pragma unroll
                for (int k = 0; k < 18; k++)
                    ((float4 *)sA)[k * NT + l] = make_float4(av[4 * k], av[4 * k + 1], av[4 * k + 2], av[4 * k + 3]);
            } else if constexpr (P == P16) {
                const uint2 *g = (const uint2 *)a.U.d;
#pragma unroll
                for (int k = 0; k < 12; k++) ((uint2 *)sU)[k * NT + l] = g[(long long)k * V + s.x];
                if constexpr (SC) {
                    const uint4 *ga = (const uint4 *)a.A.d;
#pragma unroll
                    for (int k = 0; k < 9; k++) ((uint4 *)sA)[k * NT + l] = ga[(long long)k * V + s.x];
                    sAn[l] = a.A.n[s.x];
                }
            } else {
                const float4 *g = (const float4 *)a.U.d;
#pragma unroll
                for (int k = 0; k < 12; k++) ((float4 *)sU)[k * NT + l] = g[(long long)k * V + s.x];
                if constexpr (SC) {
                    const float4 *ga = (const float4 *)a.A.d;
#pragma unroll
                    for (int k = 0; k < 18; k++) ((float4 *)sA)[k * NT + l] = ga[(long long)k * V + s.x];
                }
            }
        }
    }

    ras_mr_domain<P, NT, SC, EXP>(a, s, srho, sv, sA, lU, lA, wpart);
}

// ---------------------------------------------------------------- TMA staging
// Tensor maps of one sweep for ras_tma_kernel: every field is described as a
// 5-D tensor of 32-bit words (W words per site along x, then y, z, t, and the
// field's planes), and one box of the block's extent delivers a whole plane
// group of a domain in the kernel's shared-memory layout [plane][site].
struct RasTma {
    CUtensorMap links, clover, clover_n;
    CUtensorMap in[3], in_n[3];
    unsigned bytes;  // bytes delivered per domain by all the copies
    int nin;         // input vectors: 1, or r, v (and p) of a fused update
    // bounded-wait parameters: polls before giving up, and bytes announced on
    // top of `bytes` (non-zero only when a test makes the wait run out)
    long max_polls;
    unsigned extra_tx;
};

// The sweep of ras_smem_kernel (compact staging) for blocks without overlap
// whose extended domain has exactly NT sites, with the staging done by TMA:
// one thread issues a bulk tensor copy per plane group (links, clover, its
// norm, and each input vector with its norm), completing on an mbarrier,
// instead of every thread loading its site's 24 values through registers.
// Input vectors land in the rho/v area as raw FP16 (or FP32) planes and are
// combined (fused update) and widened there.
//
// ras_tma_body is the sweep of one (domain, right-hand side) item, with `a`
// already pointing at right-hand side rr's vectors; ras_tma_kernel runs it on
// the domains of one lattice, ras_list_kernel on a work list spanning lattices.
template <int P, int NT>
__device__ __forceinline__ void ras_tma_body(const RasArgs &a, const RasTma &tm, int rr, int dom)
{
    constexpr bool SC = P == P16;
    constexpr int RAW = P == P16 ? 52 : 96;      // bytes per site of one staged input vector
    constexpr int LW = P == P16 ? 2 : 4;         // 32-bit words per site of a link plane
    constexpr int INP = P == P16 ? 3 : 6;        // planes of an input vector
    C<float> fb, fc;
    fuse_coefs(a, rr, fb, fc);
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // 128-byte alignment for the copies, as an offset into the shared array
    // (an integer round trip would hide the address space from the compiler
    // and turn every shared-memory access into a generic one)
    unsigned char *smem = smem_dyn + ((128u - (smem_addr(smem_dyn) & 127u)) & 127u);
    __shared__ float wpart[3][NT / 32];
    __shared__ __align__(8) unsigned long long bar;
    // FP16 storage: the domain solve keeps v in tensor memory (24 columns per
    // thread; warps 4-7 of a 256-thread CTA share lanes with warps 0-3 and
    // take columns 32-55) and the links' row 2 in v's shared-memory area
    constexpr bool TMV = P == P16;
    constexpr unsigned TM_COLS = NT <= 128 ? 32u : 64u;
    __shared__ unsigned tm_base;
    float2 *srho = reinterpret_cast<float2 *>(smem);
    float2 *sv = srho + 12 * NT;
    unsigned char *sU = reinterpret_cast<unsigned char *>(sv + 12 * NT);
    unsigned char *sA = sU + (size_t)NT * RasSmem<P, false>::link_bytes;
    float *sAn = reinterpret_cast<float *>(sA + (size_t)NT * RasSmem<P, false>::clover_data);
    unsigned char *raw = smem;  // staged input vectors, inside the rho/v area
    const LinkView lU{sU};
    const CloverView lA = SC ? CloverView{sA, sAn} : a.A;
    const int l = threadIdx.x;
    LocSite s;
    loc_site(a.g, a.dg, dom, l, s);
    if (skip_domain(a, dom)) {  // uniform over the CTA, before the barrier exists
        if (s.m & M_BULK) zero_outputs<P>(a, s.x);
        return;
    }

    // the tensor-memory columns first, so that the allocation overlaps the
    // copies (allocated after the copies had landed, the 128-site sweep ran
    // 14% slower); every path below frees them
    if constexpr (TMV) {
        if (l < 32) {
            __syncwarp();  // the allocation is a warp-wide (aligned) instruction
            tm_alloc(&tm_base, TM_COLS);
        }
        tm_fence_before();
    }
    if (l == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (l == 0) {
        int k[4], r = dom;
        for (int mu = 0; mu < 4; mu++) {
            k[mu] = r % a.dg.nb[mu];
            r /= a.dg.nb[mu];
        }
        const int x0 = k[0] * a.dg.b[0], y0 = k[1] * a.dg.b[1], z0 = k[2] * a.dg.b[2], t0 = k[3] * a.dg.b[3];
        mbar_arrive_expect_tx(&bar, tm.bytes + tm.extra_tx);
        tma_load_5d(sU, &tm.links, &bar, x0 * LW, y0, z0, t0, 0);
        if constexpr (SC) {
            tma_load_5d(sA, &tm.clover, &bar, x0 * 4, y0, z0, t0, 0);
            tma_load_5d(sAn, &tm.clover_n, &bar, x0, y0, z0, t0, 0);
        }
        for (int j = 0; j < tm.nin; j++) {
            unsigned char *dst = raw + (size_t)j * RAW * NT;
            tma_load_5d(dst, &tm.in[j], &bar, x0 * 4, y0, z0, t0, rr * INP);
            if constexpr (P == P16) tma_load_5d(dst + 48 * NT, &tm.in_n[j], &bar, x0, y0, z0, t0, rr);
        }
    }
    // bounded wait, with a CTA-uniform outcome
    const bool ok = mbar_wait_bounded(&bar, 0, tm.max_polls);
    if (__syncthreads_or(!ok)) {
        if (l == 0) {
            if (a.sc) const_cast<Scalars *>(a.sc)[rr].status = S_TIMEOUT;
            else if (a.err) atomicOr(a.err, 1u);
        }
        mbar_wait_bounded(&bar, 0, tm.max_polls);  // give the copies in flight a last chance to land
        if constexpr (TMV) {
            if (l < 32) {
                __syncwarp();  // reconverge after the bounded waits
                tm_fence_after();
                tm_dealloc(tm_base, TM_COLS);
            }
        }
        return;
    }

    // the projected input: every site of a block without overlap is bulk
    C<float> r[12];
    {
        auto raw_view = [&](int j) {
            unsigned char *b = raw + (size_t)j * RAW * NT;
            return SpinorView{b, P == P16 ? reinterpret_cast<float *>(b + 48 * NT) : nullptr};
        };
        load_spinor<P>(raw_view(0), NT, l, r);
        if (tm.nin > 1) {  // fused update: inputs r, v (and p), as in staged_input
            C<float> t[12];
            load_spinor<P>(raw_view(1), NT, l, t);
#pragma unroll
            for (int q = 0; q < 12; q++) r[q] = cfma(fc, t[q], r[q]);
            if (tm.nin > 2) {
                load_spinor<P>(raw_view(2), NT, l, t);
#pragma unroll
                for (int q = 0; q < 12; q++) r[q] = cfma(fb, t[q], r[q]);
            }
        }
    }
    __syncthreads();  // all raw inputs read before rho and v overwrite them
    if constexpr (TMV) {
        tm_fence_after();
        const unsigned tv = tm_lane_addr(tm_base, (unsigned)(l >> 7) * 32u);
        st_split(srho, NT, l, r);
        const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        tm_st8(tv, z);
        tm_st8(tv + 8, z);
        tm_st8(tv + 16, z);
        stage_row2(lU, sv, (unsigned)NT, (unsigned)l);
        if (a.fuse != RAS_FUSE_NONE) store_spinor<P>(a.in, a.g.V, s.x, r);
        ras_mr_domain_x2<NT, true>(a, s, srho, sv, sA, sAn, lU, wpart, tv);
        // every warp's tensor-memory accesses are done before the release
        tm_fence_before();
        __syncthreads();
        if (l < 32) {
            __syncwarp();
            tm_fence_after();
            tm_dealloc(tm_base, TM_COLS);
        }
    } else {
        {
            C<float> z[12];
#pragma unroll
            for (int q = 0; q < 12; q++) z[q] = {0.f, 0.f};
            st_local(srho, NT, l, r);
            st_local(sv, NT, l, z);
            if (a.fuse != RAS_FUSE_NONE) store_spinor<P>(a.in, a.g.V, s.x, r);
        }
        ras_mr_domain<P, NT, SC, false>(a, s, srho, sv, sA, lU, lA, wpart);
    }
}

template <int P, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ras_tma_kernel(RasArgs a, const __grid_constant__ RasTma tm)
{
    const int rr = blockIdx.x % a.nrhs, dom = blockIdx.x / a.nrhs;
    if (a.sc && a.sc[rr].status != S_RUN) return;
    a.in = rhs_view<P>(a.in, a.g.V, rr);
    a.vout = rhs_view<P>(a.vout, a.g.V, rr);
    a.acc = rhs_view<P>(a.acc, a.g.V, rr);
    if (a.asum) a.asum += (long long)rr * 6 * a.g.V;
    ras_tma_body<P, NT>(a, tm, rr, dom);
}

// The sweeps of several lattices in one launch: a work list of (lattice,
// domain) items, lattice i owning the blocks first[i] .. first[i+1]-1, one
// domain each.  Every lattice has one right-hand side and domains of NT
// sites without overlap; blockings, N_dominv, kappa, fields and the fused
// update differ freely.  The tensor maps stay in the parameter space (their
// generic address is what the copies take); the other arguments are copied
// to shared memory once per CTA, since the lattice index is only known at
// run time.
struct RasList {
    RasTma tm[LIST_MAX];
    RasArgs a[LIST_MAX];
    int first[LIST_MAX + 1];
    int n;
};
static_assert(sizeof(RasList) <= 32000, "kernel parameter size");

template <int P, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) ras_list_kernel(const __grid_constant__ RasList L)
{
    __shared__ RasArgs sa;
    const int i = list_member(L.first, L.n);
    const RasArgs &ga = L.a[i];
    if (ga.sc[0].status != S_RUN) return;  // uniform over the CTA
    copy_words(&sa, &ga, sizeof(RasArgs));
    __syncthreads();
    ras_tma_body<P, NT>(sa, L.tm[i], 0, (int)blockIdx.x - L.first[i]);
}

// ---------------------------------------------------------------- clusters
// Extended domains too large for one CTA (overlap d > 0 on 4^4 blocks: 6^4 or
// 8^4 sites) are solved by one thread-block cluster each: one CTA per t-slice
// of the extended domain (cluster size e_t <= 8), one thread per site of the
// slice (e_x e_y e_z <= 512 sites).  Every CTA keeps its slice's residual,
// solution, links and (FP16) clover in shared memory as ras_smem_kernel does;
// the hops in t read the neighbouring slice's residual, and backwards its
// forward t link, from the neighbour CTA's shared memory (distributed shared
// memory), and the MR dot products are summed over the cluster from one
// partial per CTA.  Per MR iteration two cluster barriers order the accesses:
// one before the hops (every slice's residual is updated) and one before the
// partials are read (every hop has read the residual it needs, so it may be
// updated in place).

constexpr int RAS_CLUSTER_MAX_SLICE = 512;
constexpr int RAS_CLUSTER_MAX_CTAS = 8;

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of all CTAs of the cluster; orders shared-memory accesses
// across the cluster (release / acquire).  The split form lets a thread do
// work that needs no other CTA between its arrival and its wait.
__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync()
{
    cluster_arrive();
    cluster_wait();
}

// Arrival without ordering, for a thread whose prior writes are ordered by a
// CTA barrier and one thread's cluster-scope release fence (cluster_fence).
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_fence()
{
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
}

// Shared-memory address of p (in this CTA) mapped to CTA `rank` of the cluster.
__device__ __forceinline__ unsigned cluster_map(const void *p, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ float4 ld_cluster_f4(unsigned addr)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ uint2 ld_cluster_u2(unsigned addr)
{
    uint2 v;
    asm volatile("ld.shared::cluster.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
    return v;
}

// ld_local of site l from the residual of CTA `rank`.
__device__ __forceinline__ void ld_remote(const float2 *base, int stride, int l, unsigned rank, C<float> (&s)[12])
{
    const unsigned b = cluster_map(base, rank) + (unsigned)l * 16u;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const float4 v = ld_cluster_f4(b + (unsigned)(q * stride) * 16u);
        s[2 * q] = {v.x, v.y};
        s[2 * q + 1] = {v.z, v.w};
    }
}

// The staged forward link in direction mu of site l of CTA `rank` (the
// compact FP16 or FP32 format of the shared-memory kernel), row 2 rebuilt.
template <int P>
__device__ __forceinline__ void ld_remote_link(LinkView sU, int stride, int mu, int l, unsigned rank, C<float> (&U)[9])
{
    if constexpr (P == P32) {
        const unsigned b = cluster_map(sU.d, rank) + (unsigned)(mu * 3 * stride + l) * 16u;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const float4 a = ld_cluster_f4(b + (unsigned)(q * stride) * 16u);
            U[2 * q] = {a.x, a.y};
            U[2 * q + 1] = {a.z, a.w};
        }
    } else {
        const unsigned b = cluster_map(sU.d, rank) + (unsigned)(mu * 3 * stride + l) * 8u;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const uint2 a = ld_cluster_u2(b + (unsigned)(q * stride) * 8u);
            unsigned w[2] = {a.x, a.y};
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const float2 f2 = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
                U[2 * q + j] = {f2.x, f2.y};
            }
        }
    }
    rebuild_row2(U);
}

// The two t hops of a site whose t neighbours live in the neighbouring CTAs
// (forward: rank + 1, wrapping to 0 in a whole-lattice direction; backward:
// rank - 1, wrapping to ncta - 1).
template <int P>
__device__ __forceinline__ void cluster_hops_t(const LocSite &s, int l, const float2 *srho, LinkView sU, float kappa,
                                               C<float> (&q)[12], int NT, unsigned rank, unsigned ncta)
{
    if (s.m & (1u << 3)) {
        const unsigned nr = (s.m & (1u << 19)) ? 0u : rank + 1;
        C<float> n[12], U[9];
        ld_remote(srho, NT, l, nr, n);
        load_link<P>(sU, NT, 3, l, U);
        hop<3, true>(q, n, U, (s.m & (1u << 11)) ? kappa : -kappa);
    }
    if (s.m & (1u << 7)) {
        const unsigned nr = (s.m & (1u << 23)) ? ncta - 1 : rank - 1;
        C<float> n[12], U[9];
        ld_remote(srho, NT, l, nr, n);
        ld_remote_link<P>(sU, NT, 3, l, nr, U);
        hop<3, false>(q, n, U, (s.m & (1u << 15)) ? kappa : -kappa);
    }
}

// One cluster (dg.e[3] CTAs of blockDim.x >= e_x e_y e_z threads) per
// (domain, right-hand side); launched with the cluster dimension dg.e[3].
template <int P>
__global__ void __launch_bounds__(RAS_CLUSTER_MAX_SLICE, 1) ras_cluster_kernel(RasArgs a)
{
    constexpr bool SC = P == P16;
    const int NT = blockDim.x;
    const int S = a.dg.e[0] * a.dg.e[1] * a.dg.e[2];
    const unsigned ncta = (unsigned)a.dg.e[3];
    const unsigned rank = cluster_rank();
    const int item = blockIdx.x / ncta;
    const int rr = item % a.nrhs, dom = item / a.nrhs;
    // every decision below that returns is uniform over the cluster
    if (a.sc && a.sc[rr].status != S_RUN) return;
    a.in = rhs_view<P>(a.in, a.g.V, rr);
    a.vout = rhs_view<P>(a.vout, a.g.V, rr);
    a.acc = rhs_view<P>(a.acc, a.g.V, rr);
    a.fr = rhs_view<P>(a.fr, a.g.V, rr);
    a.fz = rhs_view<P>(a.fz, a.g.V, rr);
    if (a.asum) a.asum += (long long)rr * 6 * a.g.V;
    C<float> fb, fc;
    fuse_coefs(a, rr, fb, fc);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float wpart[3][RAS_CLUSTER_MAX_SLICE / 32];
    __shared__ float4 cpart;
    float2 *srho = reinterpret_cast<float2 *>(smem);
    float2 *sv = srho + 12 * NT;
    unsigned char *sU = reinterpret_cast<unsigned char *>(sv + 12 * NT);
    unsigned char *sA = sU + (size_t)NT * RasSmem<P, false>::link_bytes;
    float *sAn = reinterpret_cast<float *>(sA + (size_t)NT * RasSmem<P, false>::clover_data);
    const LinkView lU{sU};
    const CloverView lA = SC ? CloverView{sA, sAn} : a.A;
    const long long V = a.g.V;
    const int l = threadIdx.x;
    LocSite s;
    loc_site(a.g, a.dg, dom, l < S ? (int)rank * S + l : a.dg.nloc, s);
    const bool act = s.m & M_ACT;
    if (skip_domain(a, dom)) {
        if (s.m & M_BULK) zero_outputs<P>(a, s.x);
        return;
    }

    // stage this slice: P_{Omega'} r (or the fused update), links, clover
    {
        C<float> r[12], z[12];
#pragma unroll
        for (int k = 0; k < 12; k++) { r[k] = {0.f, 0.f}; z[k] = {0.f, 0.f}; }
        if (act) {
            staged_input<P>(a, V, s.x, fb, fc, r);
            if (a.fuse != RAS_FUSE_NONE && (s.m & M_BULK)) store_spinor<P>(a.in, V, s.x, r);
        }
        st_local(srho, NT, l, r);
        st_local(sv, NT, l, z);
        if (act) {
            if constexpr (P == P16) {
                const uint2 *g = (const uint2 *)a.U.d;
#pragma unroll
                for (int k = 0; k < 12; k++) ((uint2 *)sU)[k * NT + l] = g[(long long)k * V + s.x];
                const uint4 *ga = (const uint4 *)a.A.d;
#pragma unroll
                for (int k = 0; k < 9; k++) ((uint4 *)sA)[k * NT + l] = ga[(long long)k * V + s.x];
                sAn[l] = a.A.n[s.x];
            } else {
                const float4 *g = (const float4 *)a.U.d;
#pragma unroll
                for (int k = 0; k < 12; k++) ((float4 *)sU)[k * NT + l] = g[(long long)k * V + s.x];
            }
        }
    }

    const int nw = NT / 32;
    // The residual of this slice is staged (or, in the loop, updated): arrive
    // on the cluster barrier, make it visible to this CTA, and apply the
    // site-local and in-slice parts of D before waiting for the other slices.
    __syncthreads();
    if (l == 0) cluster_fence();
    cluster_arrive_relaxed();
    for (int it = 0; it < a.n_iter; it++) {
        C<float> q[12];
#pragma unroll
        for (int k = 0; k < 12; k++) q[k] = {0.f, 0.f};
        if (act) {
            {
                C<float> own[12];
                float av[72];
                ld_local(srho, NT, l, own);
                const float na = load_clover_u<P>(lA, SC ? (long long)NT : V, SC ? l : s.x, av);
                clover_apply(av, own, q);
                if constexpr (P == P16) {
#pragma unroll
                    for (int k = 0; k < 12; k++) q[k] = cscale(q[k], na);
                }
            }
            smem_hops<P, false, 0>(s, l, srho, lU, a.kappa, q, NT);
            smem_hops<P, false, 1>(s, l, srho, lU, a.kappa, q, NT);
            smem_hops<P, false, 2>(s, l, srho, lU, a.kappa, q, NT);
        }
        cluster_wait();  // every slice staged / updated
        if (act) cluster_hops_t<P>(s, l, srho, lU, a.kappa, q, NT, rank, ncta);
        // <q, rho> and |q|^2: warps, then the CTA (thread 0), then the cluster
        float red[3];
        {
            C<float> own[12];
            ld_local(srho, NT, l, own);
            float qr = 0.f, qi = 0.f, qq = 0.f;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                cdot_acc(q[k], own[k], qr, qi);
                cnorm_acc(q[k], qq);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                qr += __shfl_xor_sync(0xffffffffu, qr, o);
                qi += __shfl_xor_sync(0xffffffffu, qi, o);
                qq += __shfl_xor_sync(0xffffffffu, qq, o);
            }
            if ((l & 31) == 0) {
                wpart[0][l >> 5] = qr;
                wpart[1][l >> 5] = qi;
                wpart[2][l >> 5] = qq;
            }
            __syncthreads();
            if (l == 0) {
                float4 t = {0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < nw; w++) {
                    t.x += wpart[0][w];
                    t.y += wpart[1][w];
                    t.z += wpart[2][w];
                }
                cpart = t;
                cluster_fence();
            }
            // every partial written (thread 0's fence releases it); every hop
            // has read its residual (the loaded values are consumed already)
            cluster_arrive_relaxed();
            cluster_wait();
            const int lane = l & 31;
            float4 t = {0.f, 0.f, 0.f, 0.f};
            if (lane < (int)ncta) t = ld_cluster_f4(cluster_map(&cpart, (unsigned)lane));
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
                t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
                t.z += __shfl_xor_sync(0xffffffffu, t.z, o);
            }
            // lane 0's sum, identical in every warp of every CTA
            red[0] = __shfl_sync(0xffffffffu, t.x, 0);
            red[1] = __shfl_sync(0xffffffffu, t.y, 0);
            red[2] = __shfl_sync(0xffffffffu, t.z, 0);
        }
        if (red[2] > 0.f) {
            const float inv = 1.0f / red[2];
            const C<float> al = {red[0] * inv, red[1] * inv};
            C<float> own[12], vv[12];
            ld_local(srho, NT, l, own);
            ld_local(sv, NT, l, vv);
#pragma unroll
            for (int k = 0; k < 12; k++) {
                vv[k] = cfma(al, own[k], vv[k]);
                own[k] = cfma(cneg(al), q[k], own[k]);
            }
            st_local(sv, NT, l, vv);
            st_local(srho, NT, l, own);
        }
        // the updated residual: visible to this CTA after the CTA barrier, to
        // the cluster after thread 0's release fence that follows it
        __syncthreads();
        if (l == 0) cluster_fence();
        cluster_arrive_relaxed();
    }
    // no CTA leaves while another may still read its partial or residual
    cluster_wait();
    if (a.asum) {
        if (act) {
            C<float> vv[12];
            ld_local(sv, NT, l, vv);
            as_add(a, s.x, vv);
        }
    } else if (s.m & M_BULK) {
        C<float> vv[12];
        ld_local(sv, NT, l, vv);
        write_outputs<P>(a, s.x, vv);
    }
}

constexpr int RAS_GMEM_NT = 256;

template <int P>
__global__ void __launch_bounds__(RAS_GMEM_NT) ras_gmem_kernel(const RasArgs a0)
{
    __shared__ double red_sm[3 * 32 + 3];
    const int n = a0.dg.nloc;
    float2 *rho = a0.scratch + (size_t)blockIdx.x * 36 * n;
    float2 *q = rho + 12 * (size_t)n;
    float2 *vv = q + 12 * (size_t)n;
    // work items are (domain, right-hand side) pairs, right-hand side fastest
    for (int item = blockIdx.x; item < a0.dg.ndom * a0.nrhs; item += gridDim.x) {
        const int dom = item / a0.nrhs, rr = item % a0.nrhs;
        if (a0.sc && a0.sc[rr].status != S_RUN) continue;  // uniform over the CTA
        RasArgs a = a0;
        a.in = rhs_view<P>(a0.in, a0.g.V, rr);
        a.vout = rhs_view<P>(a0.vout, a0.g.V, rr);
        a.acc = rhs_view<P>(a0.acc, a0.g.V, rr);
        if (a.asum) a.asum += (long long)rr * 6 * a.g.V;
        if (skip_domain(a, dom)) {  // uniform over the CTA
            for (int l = threadIdx.x; l < n; l += RAS_GMEM_NT) {
                DomSite ds;
                dom_site(a.g, a.dg, dom, l, a.kappa, ds);
                if (ds.bulk) zero_outputs<P>(a, ds.x);
            }
            continue;
        }
        for (int l = threadIdx.x; l < n; l += RAS_GMEM_NT) {
            DomSite ds;
            dom_site(a.g, a.dg, dom, l, a.kappa, ds);
            C<float> r[12], z[12];
            load_spinor<P>(a.in, a.g.V, ds.x, r);
#pragma unroll
            for (int k = 0; k < 12; k++) z[k] = {0.f, 0.f};
            st_local(rho, n, l, r);
            st_local(vv, n, l, z);
        }
        for (int it = 0; it < a.n_iter; it++) {
            __syncthreads();
            double red[3] = {0.0, 0.0, 0.0};
            for (int l = threadIdx.x; l < n; l += RAS_GMEM_NT) {
                DomSite ds;
                dom_site(a.g, a.dg, dom, l, a.kappa, ds);
                C<float> own[12], qq[12];
                ld_local(rho, n, l, own);
                dom_apply<P>(a, ds, own, rho, n, qq);
                st_local(q, n, l, qq);
                float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    cdot_acc(qq[k], own[k], s0, s1);
                    cnorm_acc(qq[k], s2);
                }
                red[0] += s0;
                red[1] += s1;
                red[2] += s2;
            }
            block_allsum<3>(red, red_sm);
            if (red[2] > 0.0) {
                const C<float> al = {(float)(red[0] / red[2]), (float)(red[1] / red[2])};
                for (int l = threadIdx.x; l < n; l += RAS_GMEM_NT) {
#pragma unroll
                    for (int k = 0; k < 12; k++) {
                        float2 r2 = rho[k * n + l], q2 = q[k * n + l], v2 = vv[k * n + l];
                        C<float> r = {r2.x, r2.y}, qc = {q2.x, q2.y}, vc = {v2.x, v2.y};
                        vc = cfma(al, r, vc);
                        r = cfma(cneg(al), qc, r);
                        rho[k * n + l] = make_float2(r.r, r.i);
                        vv[k * n + l] = make_float2(vc.r, vc.i);
                    }
                }
            }
        }
        __syncthreads();
        for (int l = threadIdx.x; l < n; l += RAS_GMEM_NT) {
            DomSite ds;
            dom_site(a.g, a.dg, dom, l, a.kappa, ds);
            if (a.asum) {
                C<float> v[12];
                ld_local(vv, n, l, v);
                as_add(a, ds.x, v);
            } else if (ds.bulk) {
                C<float> v[12];
                ld_local(vv, n, l, v);
                write_outputs<P>(a, ds.x, v);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- phased
// Few large domains (the paper's slabs: 8 domains of 4 x 32^3 sites and
// more) leave most SMs idle with one CTA per domain.  The phased sweep spreads
// every domain over many CTAs and runs the MR iterations as launches: stage
// (rho = P r, v = 0), then per iteration apply (q = D_Omega' rho and one
// partial of <q, rho>, |q|^2 per CTA), alpha (one CTA per domain adds the
// partials in CTA order) and update (v += alpha rho, rho -= alpha q), and
// finally the restriction.  rho, q and v live in a global-scratch slot per
// (domain, right-hand side) as for ras_gmem_kernel; kernel boundaries order
// the iterations.  Items are (domain, right-hand side) pairs, right-hand side
// fastest; CTA b works on chunk b / items of item b % items, so that the CTAs
// running together cover the same local sites of every domain: neighbouring
// slabs share the cache lines of the fields (a 4-site-wide slab uses half of
// each 128-byte line of a plane), which are then fetched once.

constexpr int RAS_PH_NT = 256;

struct PhaseGrid {
    int nblk;  // CTAs per item
};

__device__ __forceinline__ float2 *phase_slot(const RasArgs &a, int item)
{
    return a.scratch + (size_t)item * 36 * (size_t)a.dg.nloc;
}

// the partial sums (3 per CTA) and the alphas (one float2 per item, 16-byte
// aligned) after the slots
__device__ __forceinline__ float *phase_partials(const RasArgs &a, int items)
{
    return reinterpret_cast<float *>(a.scratch + (size_t)items * 36 * (size_t)a.dg.nloc);
}

__device__ __forceinline__ float2 *phase_alpha(const RasArgs &a, int items, int nblk)
{
    const size_t off = ((size_t)items * nblk * 3 + 3) & ~(size_t)3;
    return reinterpret_cast<float2 *>(phase_partials(a, items) + off);
}

template <int P>
__device__ __forceinline__ bool phase_item(RasArgs &a, int item, int &dom, int &rr)
{
    rr = item % a.nrhs;
    dom = item / a.nrhs;
    if (a.sc && a.sc[rr].status != S_RUN) return false;
    a.in = rhs_view<P>(a.in, a.g.V, rr);
    a.vout = rhs_view<P>(a.vout, a.g.V, rr);
    a.acc = rhs_view<P>(a.acc, a.g.V, rr);
    if (a.asum) a.asum += (long long)rr * 6 * a.g.V;
    return true;
}

template <int P>
__global__ void __launch_bounds__(RAS_PH_NT) ras_phase_stage(RasArgs a, PhaseGrid pg)
{
    const int items = gridDim.x / pg.nblk;
    const int item = blockIdx.x % items, chunk = blockIdx.x / items;
    int dom, rr;
    if (!phase_item<P>(a, item, dom, rr) || skip_domain(a, dom)) return;
    const int n = a.dg.nloc, l = chunk * RAS_PH_NT + threadIdx.x;
    if (l >= n) return;
    float2 *rho = phase_slot(a, item), *v = rho + 24 * (size_t)n;
    DomSite ds;
    dom_site(a.g, a.dg, dom, l, a.kappa, ds);
    C<float> r[12], z[12];
    load_spinor<P>(a.in, a.g.V, ds.x, r);
#pragma unroll
    for (int k = 0; k < 12; k++) z[k] = {0.f, 0.f};
    st_local(rho, n, l, r);
    st_local(v, n, l, z);
}

template <int P>
__global__ void __launch_bounds__(RAS_PH_NT) ras_phase_apply(RasArgs a, PhaseGrid pg, int items)
{
    __shared__ double sm[3 * 32];
    const int item = blockIdx.x % items, chunk = blockIdx.x / items;
    int dom, rr;
    if (!phase_item<P>(a, item, dom, rr) || skip_domain(a, dom)) return;  // uniform over the CTA
    const int n = a.dg.nloc, l = chunk * RAS_PH_NT + threadIdx.x;
    float2 *rho = phase_slot(a, item), *q = rho + 12 * (size_t)n;
    float part[3] = {0.f, 0.f, 0.f};
    if (l < n) {
        DomSite ds;
        dom_site(a.g, a.dg, dom, l, a.kappa, ds);
        C<float> own[12], qq[12];
        ld_local(rho, n, l, own);
        dom_apply<P>(a, ds, own, rho, n, qq);
        st_local(q, n, l, qq);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            cdot_acc(qq[k], own[k], part[0], part[1]);
            cnorm_acc(qq[k], part[2]);
        }
    }
    double red[3];
    block_sum<3, float>(part, red, sm);
    if (threadIdx.x == 0) {
        float *pp = phase_partials(a, items) + ((size_t)item * pg.nblk + chunk) * 3;
        pp[0] = (float)red[0];
        pp[1] = (float)red[1];
        pp[2] = (float)red[2];
    }
}

template <int P>
__global__ void __launch_bounds__(RAS_PH_NT) ras_phase_alpha(RasArgs a, PhaseGrid pg, int items)
{
    __shared__ double sm[3 * 32 + 3];
    const int item = blockIdx.x;
    int dom, rr;
    if (!phase_item<P>(a, item, dom, rr) || skip_domain(a, dom)) return;
    const float *pp = phase_partials(a, items) + (size_t)item * pg.nblk * 3;
    double red[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < pg.nblk; b += RAS_PH_NT) {
        red[0] += pp[3 * b];
        red[1] += pp[3 * b + 1];
        red[2] += pp[3 * b + 2];
    }
    block_sum<3>(red, sm);
    if (threadIdx.x == 0) {
        float2 *alpha = phase_alpha(a, items, pg.nblk);
        alpha[item] = red[2] > 0.0 ? make_float2((float)(red[0] / red[2]), (float)(red[1] / red[2]))
                                   : make_float2(0.f, 0.f);
    }
}

template <int P>
__global__ void __launch_bounds__(RAS_PH_NT) ras_phase_update(RasArgs a, PhaseGrid pg, int items)
{
    const int item = blockIdx.x % items, chunk = blockIdx.x / items;
    int dom, rr;
    if (!phase_item<P>(a, item, dom, rr) || skip_domain(a, dom)) return;
    const int n = a.dg.nloc, l = chunk * RAS_PH_NT + threadIdx.x;
    if (l >= n) return;
    const float2 al2 = phase_alpha(a, items, pg.nblk)[item];
    const C<float> al = {al2.x, al2.y};
    float2 *rho = phase_slot(a, item), *q = rho + 12 * (size_t)n, *v = rho + 24 * (size_t)n;
    C<float> r[12], qq[12], vv[12];
    ld_local(rho, n, l, r);
    ld_local(q, n, l, qq);
    ld_local(v, n, l, vv);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        vv[k] = cfma(al, r[k], vv[k]);
        r[k] = cfma(cneg(al), qq[k], r[k]);
    }
    st_local(v, n, l, vv);
    st_local(rho, n, l, r);
}

template <int P>
__global__ void __launch_bounds__(RAS_PH_NT) ras_phase_output(RasArgs a, PhaseGrid pg)
{
    const int items = gridDim.x / pg.nblk;
    const int item = blockIdx.x % items, chunk = blockIdx.x / items;
    int dom, rr;
    if (!phase_item<P>(a, item, dom, rr)) return;
    const int n = a.dg.nloc, l = chunk * RAS_PH_NT + threadIdx.x;
    if (l >= n) return;
    DomSite ds;
    dom_site(a.g, a.dg, dom, l, a.kappa, ds);
    if (skip_domain(a, dom)) {
        if (ds.bulk) zero_outputs<P>(a, ds.x);
        return;
    }
    const float2 *v = phase_slot(a, item) + 24 * (size_t)n;
    if (a.asum) {
        C<float> vv[12];
        ld_local(v, n, l, vv);
        as_add(a, ds.x, vv);
    } else if (ds.bulk) {
        C<float> vv[12];
        ld_local(v, n, l, vv);
        write_outputs<P>(a, ds.x, vv);
    }
}

// The phased sweep is used when the domains (times right-hand sides) are
// too few to fill the GPU with one CTA each.
bool ras_use_phased(const DomainGeom &dg, int nrhs)
{
    return dg.nloc > RAS_SMEM_MAX_SITES && (long long)dg.ndom * nrhs < 2 * 152 && !ras_cluster_shape(dg);
}

size_t ras_phased_scratch_bytes(const DomainGeom &dg, int nrhs)
{
    const long long items = (long long)dg.ndom * nrhs;
    const long long nblk = (dg.nloc + RAS_PH_NT - 1) / RAS_PH_NT;
    return (size_t)items * 36 * (size_t)dg.nloc * sizeof(float2) +
           (size_t)((items * nblk * 3 + 3) & ~3LL) * sizeof(float) + (size_t)items * sizeof(float2);
}

template <int P>
static cudaError_t launch_phased(const RasArgs &a, cudaStream_t st)
{
    if (a.fuse != RAS_FUSE_NONE || !a.scratch) return cudaErrorInvalidValue;
    const int items = a.dg.ndom * a.nrhs;
    PhaseGrid pg;
    pg.nblk = (a.dg.nloc + RAS_PH_NT - 1) / RAS_PH_NT;
    const unsigned grid = (unsigned)((long long)items * pg.nblk);
    ras_phase_stage<P><<<grid, RAS_PH_NT, 0, st>>>(a, pg);
    note_launch();
    for (int it = 0; it < a.n_iter; it++) {
        ras_phase_apply<P><<<grid, RAS_PH_NT, 0, st>>>(a, pg, items);
        ras_phase_alpha<P><<<items, RAS_PH_NT, 0, st>>>(a, pg, items);
        ras_phase_update<P><<<grid, RAS_PH_NT, 0, st>>>(a, pg, items);
        note_launch(3);
    }
    ras_phase_output<P><<<grid, RAS_PH_NT, 0, st>>>(a, pg);
    note_launch();
    return cudaGetLastError();
}

template <int P, int NT, bool SC, bool EXP = false>
static cudaError_t launch_smem(const RasArgs &a, cudaStream_t st)
{
    const size_t smem = RasSmem<P, EXP>::bytes(NT, SC || EXP);
    // the shared-memory opt-in is set once per device (before any capture:
    // the first launch of a solve is never captured)
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !((done.load() >> dev) & 1ull)) {
        cudaError_t e = cudaFuncSetAttribute(ras_smem_kernel<P, NT, SC || EXP, EXP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done.fetch_or(1ull << dev);
    }
    ras_smem_kernel<P, NT, SC || EXP, EXP><<<a.dg.ndom * a.nrhs, NT, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

// Domains of up to 128 sites use the expanded staging (FP32 18-real links and
// FP32 clover, 768 B per site); 256-site domains keep the links 12-real and,
// for FP16 storage, the clover in FP16 (111.6 KB, two CTAs per SM); for FP32
// storage the clover is read through L1 instead.
// ---------------------------------------------------------------- TMA host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no
// link-time dependency on the driver library); null if unavailable.
static EncodeTiledFn tma_encoder()
{
    static std::atomic<int> state{0};  // 0 unknown, 1 found, 2 unavailable
    static EncodeTiledFn fn = nullptr;
    int s = state.load();
    if (s == 0) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && f) {
            fn = reinterpret_cast<EncodeTiledFn>(f);
            state.store(1);
        } else {
            cudaGetLastError();
            state.store(2);
        }
        s = state.load();
    }
    return s == 1 ? fn : nullptr;
}

// Map of a planar field with w 32-bit words per site and `planes` planes of V
// sites, boxed by the block (b) and `box_planes` planes.
static bool encode_field(EncodeTiledFn enc, CUtensorMap *m, const void *base, int w, const Geom &g, long long planes,
                         const int b[4], int box_planes, unsigned *bytes)
{
    if (!base || (reinterpret_cast<size_t>(base) & 15)) return false;
    const cuuint64_t row = (cuuint64_t)w * 4 * g.L[0];
    const cuuint64_t dims[5] = {(cuuint64_t)w * g.L[0], (cuuint64_t)g.L[1], (cuuint64_t)g.L[2], (cuuint64_t)g.L[3],
                                (cuuint64_t)planes};
    const cuuint64_t strides[4] = {row, row * g.L[1], row * g.L[1] * g.L[2], (cuuint64_t)w * 4 * g.V};
    const cuuint32_t box[5] = {(cuuint32_t)(w * b[0]), (cuuint32_t)b[1], (cuuint32_t)b[2], (cuuint32_t)b[3],
                               (cuuint32_t)box_planes};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    for (int i = 0; i < 4; i++)
        if (strides[i] % 16 || strides[i] >= (1ull << 40)) return false;
    for (int i = 0; i < 5; i++)
        if (box[i] < 1 || box[i] > 256 || box[i] > dims[i]) return false;
    if ((box[0] * 4) % 16) return false;
    if (enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    *bytes += box[0] * box[1] * box[2] * box[3] * box[4] * 4u;
    return true;
}

// Bounded-wait settings of the TMA sweep (see qdd_test_ras_wait).
static std::atomic<long> g_tma_polls{TMA_WAIT_TRIES};
static std::atomic<unsigned> g_tma_extra_tx{0};

void ras_set_wait_test(unsigned extra_bytes, long max_polls)
{
    g_tma_extra_tx.store(extra_bytes);
    g_tma_polls.store(max_polls > 0 ? max_polls : TMA_WAIT_TRIES);
}

// Builds the maps of ras_tma_kernel for this sweep; false when the sweep does
// not qualify (overlap, domain size, extents not multiples of 4 along x,
// misaligned fields, a fused p update in FP32, no encoder).
template <int P>
static bool tma_maps(const RasArgs &a, int nt, RasTma *tm)
{
    if (a.variant != 0 || a.dg.nloc != nt) return false;
    for (int mu = 0; mu < 4; mu++)
        if (a.dg.e[mu] != a.dg.b[mu]) return false;
    if (a.dg.b[0] % 4 || a.g.L[0] % 4) return false;
    if (P == P32 && a.fuse == RAS_FUSE_P) return false;
    EncodeTiledFn enc = tma_encoder();
    if (!enc) return false;
    memset(tm, 0, sizeof(*tm));
    tm->max_polls = g_tma_polls.load();
    tm->extra_tx = g_tma_extra_tx.load();
    const int lw = P == P16 ? 2 : 4, inp = P == P16 ? 3 : 6;
    if (!encode_field(enc, &tm->links, a.U.d, lw, a.g, 12, a.dg.b, 12, &tm->bytes)) return false;
    if (P == P16) {
        if (!encode_field(enc, &tm->clover, a.A.d, 4, a.g, 9, a.dg.b, 9, &tm->bytes)) return false;
        if (!encode_field(enc, &tm->clover_n, a.A.n, 1, a.g, 1, a.dg.b, 1, &tm->bytes)) return false;
    }
    const SpinorView ins[3] = {a.fuse == RAS_FUSE_NONE ? a.in : a.fr, a.fz, a.in};
    tm->nin = a.fuse == RAS_FUSE_NONE ? 1 : a.fuse == RAS_FUSE_S ? 2 : 3;
    for (int j = 0; j < tm->nin; j++) {
        if (!encode_field(enc, &tm->in[j], ins[j].d, 4, a.g, (long long)inp * a.nrhs, a.dg.b, inp, &tm->bytes))
            return false;
        if (P == P16 && !encode_field(enc, &tm->in_n[j], ins[j].n, 1, a.g, a.nrhs, a.dg.b, 1, &tm->bytes))
            return false;
    }
    return true;
}

template <int P, int NT>
static cudaError_t launch_tma(const RasArgs &a, const RasTma &tm, cudaStream_t st)
{
    const size_t smem = RasSmem<P, false>::bytes(NT, P == P16) + 128;
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !((done.load() >> dev) & 1ull)) {
        cudaError_t e =
            cudaFuncSetAttribute(ras_tma_kernel<P, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done.fetch_or(1ull << dev);
    }
    ras_tma_kernel<P, NT><<<a.dg.ndom * a.nrhs, NT, smem, st>>>(a, tm);
    note_launch();
    return cudaGetLastError();
}

template <int P>
static bool ras_list_ok_p(const RasArgs &a)
{
    const int n = a.dg.nloc;
    if ((n != 128 && n != 256) || a.nrhs != 1 || !a.sc || a.asum || a.color != 0) return false;
    RasTma tm;
    return tma_maps<P>(a, n, &tm);
}

bool ras_list_ok(int prec, const RasArgs &a) { return prec == P16 && ras_list_ok_p<P16>(a); }

template <int P, int NT>
static cudaError_t launch_list_nt(const RasArgs *as, int n, cudaStream_t st)
{
    const size_t smem = RasSmem<P, false>::bytes(NT, P == P16) + 128;
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !((done.load() >> dev) & 1ull)) {
        cudaError_t e =
            cudaFuncSetAttribute(ras_list_kernel<P, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done.fetch_or(1ull << dev);
    }
    // one parameter block, built on the host per launch (a captured graph
    // keeps its own copy)
    static thread_local RasList L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    long long total = 0;
    for (int i = 0; i < n; i++) {
        if (as[i].dg.nloc != NT || !ras_list_ok_p<P>(as[i]) || !tma_maps<P>(as[i], NT, &L.tm[i]))
            return cudaErrorInvalidValue;
        L.a[i] = as[i];
        L.first[i] = (int)total;
        total += as[i].dg.ndom;
    }
    L.first[n] = (int)total;
    if (total >= (1LL << 31)) return cudaErrorInvalidConfiguration;
    ras_list_kernel<P, NT><<<(unsigned)total, NT, smem, st>>>(L);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ras_list(int prec, const RasArgs *as, int n, cudaStream_t st)
{
    if (n < 1 || n > LIST_MAX) return cudaErrorInvalidValue;
    if (prec != P16) return cudaErrorInvalidValue;
    return as[0].dg.nloc == 256 ? launch_list_nt<P16, 256>(as, n, st) : launch_list_nt<P16, 128>(as, n, st);
}

// vout = asum, acc = asum (or acc += asum) on every site: the additive
// Schwarz sum of one sweep, in the fields' precision.  grid.y = right-hand side.
template <int P>
__global__ void __launch_bounds__(256) as_finish_kernel(const RasArgs a)
{
    const int rr = blockIdx.y;
    if (a.sc && a.sc[rr].status != S_RUN) return;
    const long long V = a.g.V;
    const long long x = (long long)blockIdx.x * 256 + threadIdx.x;
    if (x >= V) return;
    const float4 *sum = a.asum + (long long)rr * 6 * V;
    C<float> v[12];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const float4 f = sum[(long long)k * V + x];
        v[2 * k] = {f.x, f.y};
        v[2 * k + 1] = {f.z, f.w};
    }
    write_outputs_to<P>(rhs_view<P>(a.vout, V, rr), rhs_view<P>(a.acc, V, rr), a.accumulate, V, x, v);
}

cudaError_t launch_as_finish(int prec, const RasArgs &a, cudaStream_t st)
{
    if (!a.asum || a.nrhs < 1 || a.nrhs > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((a.g.V + 255) / 256), (unsigned)a.nrhs);
    switch (prec) {
    case P32: as_finish_kernel<P32><<<grid, 256, 0, st>>>(a); break;
    case P16: as_finish_kernel<P16><<<grid, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

bool ras_cluster_shape(const DomainGeom &dg)
{
    const int slice = dg.e[0] * dg.e[1] * dg.e[2];
    return dg.nloc > RAS_SMEM_MAX_SITES && dg.e[3] >= 2 && dg.e[3] <= RAS_CLUSTER_MAX_CTAS &&
           slice <= RAS_CLUSTER_MAX_SLICE;
}

// Launches ras_cluster_kernel when the device can hold one of its clusters
// (*launched = true); otherwise launches nothing and the caller falls back to
// the general kernel.  The shared-memory opt-in and the residency query are
// made once per device and cluster shape (before any capture: the first
// launch of a solve is never captured).
template <int P>
static cudaError_t launch_cluster(const RasArgs &a, cudaStream_t st, bool *launched)
{
    *launched = false;
    const int slice = a.dg.e[0] * a.dg.e[1] * a.dg.e[2];
    const int ncta = a.dg.e[3];
    const int nt = (slice + 31) / 32 * 32;
    const size_t smem = RasSmem<P, false>::bytes(nt, P == P16);
    int dev = 0;
    cudaGetDevice(&dev);
    // per device: bit 0 opt-in done; per (cluster size, warps) a residency
    // state 0 unknown, 1 resident, 2 not resident
    static std::atomic<unsigned> optin[64];
    static std::atomic<unsigned char> state[64][RAS_CLUSTER_MAX_CTAS + 1][RAS_CLUSTER_MAX_SLICE / 32 + 1];
    if (dev < 0 || dev >= 64) return cudaSuccess;
    if (!(optin[dev].load() & 1u)) {
        cudaError_t e = cudaFuncSetAttribute(ras_cluster_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)RasSmem<P, false>::bytes(RAS_CLUSTER_MAX_SLICE, P == P16));
        if (e != cudaSuccess) return e;
        optin[dev].fetch_or(1u);
    }
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)((long long)ncta * a.dg.ndom * a.nrhs), 1, 1);
    cfg.blockDim = dim3((unsigned)nt, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    std::atomic<unsigned char> &known = state[dev][ncta][nt / 32];
    if (known.load() == 0) {
        int clusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, ras_cluster_kernel<P>, &cfg);
        if (e != cudaSuccess) {
            cudaGetLastError();
            clusters = 0;
        }
        known.store(clusters > 0 ? 1 : 2);
    }
    if (known.load() != 1) return cudaSuccess;
    cudaError_t e = cudaLaunchKernelEx(&cfg, ras_cluster_kernel<P>, a);
    note_launch();
    *launched = true;
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int P>
static cudaError_t launch_p(const RasArgs &a, cudaStream_t st)
{
    const int n = a.dg.nloc;
    if constexpr (P == P16 || P == P32) {
        // (the TMA kernel serves blocks without overlap, where the additive
        // sum is never used)
        if ((n == 256 || n == 128) && !a.asum) {
            RasTma tm;
            if (tma_maps<P>(a, n, &tm)) return n == 256 ? launch_tma<P, 256>(a, tm, st) : launch_tma<P, 128>(a, tm, st);
        }
        if (a.variant == 1) {  // compact staging at every size
            if (n <= 32) return launch_smem<P, 32, P == P16>(a, st);
            if (n <= 64) return launch_smem<P, 64, P == P16>(a, st);
            if (n <= 128) return launch_smem<P, 128, P == P16>(a, st);
        }
        if (a.variant == 2 && n > 128 && n <= 256) return launch_smem<P, 256, true, true>(a, st);
        if (n <= 32) return launch_smem<P, 32, true, true>(a, st);
        if (n <= 64) return launch_smem<P, 64, true, true>(a, st);
        if (n <= 128) return launch_smem<P, 128, true, true>(a, st);
        if (n <= 256) return launch_smem<P, 256, P == P16>(a, st);
        if (n <= RAS_SMEM_MAX_SITES) return launch_smem<P, 512, P == P16>(a, st);
    }
    if constexpr (P == P16 || P == P32) {
        if (a.variant != 3 && a.fuse == RAS_FUSE_NONE && ras_cluster_shape(a.dg)) {
            bool ok = false;
            const cudaError_t e = launch_cluster<P>(a, st, &ok);
            if (ok || e != cudaSuccess) return e;
        }
    }
    if constexpr (P == P16 || P == P32) {
        if (a.variant != 3 && ras_use_phased(a.dg, a.nrhs)) return launch_phased<P>(a, st);
    }
    // the general kernel has no fused update (the caller checks ras_can_fuse)
    if (a.fuse != RAS_FUSE_NONE || !a.scratch || a.slots < 1) return cudaErrorInvalidValue;
    const long long items = (long long)a.dg.ndom * a.nrhs;
    const int grid = a.slots < items ? a.slots : (int)items;
    ras_gmem_kernel<P><<<grid, RAS_GMEM_NT, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ras_block(int prec, const RasArgs &a, cudaStream_t st)
{
    if (a.dg.ndom <= 0) return cudaSuccess;
    if (a.nrhs < 1) return cudaErrorInvalidValue;
    switch (prec) {
    case P64: return launch_p<P64>(a, st);
    case P32: return launch_p<P32>(a, st);
    case P16: return launch_p<P16>(a, st);
    }
    return cudaErrorInvalidValue;
}

template <int P>
static cudaError_t launch_gmem_p(const RasArgs &a, cudaStream_t st)
{
    // the general kernel has no fused update (the caller checks ras_can_fuse)
    if (a.fuse != RAS_FUSE_NONE || !a.scratch || a.slots < 1) return cudaErrorInvalidValue;
    const long long items = (long long)a.dg.ndom * a.nrhs;
    const int grid = a.slots < items ? a.slots : (int)items;
    ras_gmem_kernel<P><<<grid, RAS_GMEM_NT, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ras_block_gmem(int prec, const RasArgs &a, cudaStream_t st)
{
    if (a.dg.ndom <= 0) return cudaSuccess;
    if (a.nrhs < 1) return cudaErrorInvalidValue;
    switch (prec) {
    case P32: return launch_gmem_p<P32>(a, st);
    case P16: return launch_gmem_p<P16>(a, st);
    }
    return cudaErrorInvalidValue;
}

int ras_default_slots() { return 2 * 152; }

size_t ras_scratch_bytes(const DomainGeom &dg, int slots, int nrhs)
{
    if (dg.nloc <= RAS_SMEM_MAX_SITES) return 0;
    const long long items = (long long)dg.ndom * nrhs;
    const int s = slots < items ? slots : (int)items;
    const size_t gmem = (size_t)s * 36 * (size_t)dg.nloc * sizeof(float2);
    // the phased sweep needs a slot per item plus its partial sums
    if (ras_use_phased(dg, nrhs)) {
        const size_t ph = ras_phased_scratch_bytes(dg, nrhs);
        return ph > gmem ? ph : gmem;
    }
    return gmem;
}

bool domain_geom(const Geom &g, const int block[4], int s, DomainGeom *dg, std::string *why)
{
    if (s < 0) {
        if (why) *why = "overlap must be >= 0";
        return false;
    }
    dg->ndom = 1;
    long long nloc = 1;
    for (int mu = 0; mu < 4; mu++) {
        const int b = block[mu], L = g.L[mu];
        if (b <= 0 || L % b != 0) {
            if (why) *why = "block[" + std::to_string(mu) + "] = " + std::to_string(b) + " does not divide L = " +
                            std::to_string(L);
            return false;
        }
        dg->b[mu] = b;
        if (b == L) {
            dg->e[mu] = L;
            dg->sh[mu] = 0;
        } else {
            if (b + 2 * s > L) {
                if (why) *why = "block + 2*overlap exceeds the lattice in direction " + std::to_string(mu);
                return false;
            }
            dg->e[mu] = b + 2 * s;
            dg->sh[mu] = s;
        }
        dg->nb[mu] = L / b;
        dg->ndom *= dg->nb[mu];
        nloc *= dg->e[mu];
    }
    if (nloc > (1LL << 30)) {
        if (why) *why = "extended domain too large";
        return false;
    }
    dg->nloc = (int)nloc;
    for (int mu = 0; mu < 4; mu++) {
        division_magic(dg->nb[mu], &dg->nb_m[mu], &dg->nb_sh[mu]);
        division_magic(dg->e[mu], &dg->e_m[mu], &dg->e_sh[mu]);
    }
    return true;
}

}  // namespace qdd
