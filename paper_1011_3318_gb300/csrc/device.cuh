// device.cuh -- device building blocks of the Wilson-clover operator.
//
// The operator (Eq. 1 of Osaki & Ishikawa, Lattice 2010, with the O(a)
// improvement of Sec. 5) is D = A - kappa H, where the hop in direction mu
// carries the spin projector (1 - gamma_mu) forward and (1 + gamma_mu)
// backward.  In the DeGrand-Rossi basis every gamma_mu is off-diagonal in
// chirality, gamma_mu = [[0, X_mu], [X_mu^dag, 0]] on (upper spins 0,1 ;
// lower spins 2,3), with
//     X_x = [[0, i], [i, 0]],   X_y = [[0, -1], [1, 0]],
//     X_z = [[i, 0], [0, -i]],  X_t = 1.
// Hence (1 -+ gamma_mu) psi = [h ; -+ X_mu^dag h] with h = up -+ X_mu dn: only
// the two-spin half spinor h is multiplied by the link, and the lower half
// is rebuilt from it.  This file derives its constants from that structure
// alone.
#pragma once

#include <cuda_fp16.h>

#include "qdd_internal.h"

namespace qdd {

template <int P> struct RealOf { typedef float T; };
template <> struct RealOf<P64> { typedef double T; };

template <typename T> struct C { T r, i; };

template <typename T> __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T> __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T> __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b)
{
    return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
// conj(a) * b
template <typename T> __device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b)
{
    return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r};
}
// c + a b and c + conj(a) b as chains of four fused multiply-adds: written
// as cadd(c, cmul(a, b)) the compiler, which does not reassociate, emits two
// multiplies, two fused multiply-adds and two adds.
template <typename T> __device__ __forceinline__ C<T> cfma(C<T> a, C<T> b, C<T> c)
{
    c.r = fma(a.r, b.r, c.r);
    c.r = fma(-a.i, b.i, c.r);
    c.i = fma(a.r, b.i, c.i);
    c.i = fma(a.i, b.r, c.i);
    return c;
}
template <typename T> __device__ __forceinline__ C<T> cfmac(C<T> a, C<T> b, C<T> c)
{
    c.r = fma(a.r, b.r, c.r);
    c.r = fma(a.i, b.i, c.r);
    c.i = fma(a.r, b.i, c.i);
    c.i = fma(-a.i, b.r, c.i);
    return c;
}
// (re, im) += conj(a) b and n += |a|^2, also as fused multiply-add chains
template <typename T> __device__ __forceinline__ void cdot_acc(C<T> a, C<T> b, T &re, T &im)
{
    re = fma(a.r, b.r, re);
    re = fma(a.i, b.i, re);
    im = fma(a.r, b.i, im);
    im = fma(-a.i, b.r, im);
}
template <typename T> __device__ __forceinline__ void cnorm_acc(C<T> a, T &n)
{
    n = fma(a.r, a.r, n);
    n = fma(a.i, a.i, n);
}
template <typename T> __device__ __forceinline__ C<T> cscale(C<T> a, T s) { return {a.r * s, a.i * s}; }
template <typename T> __device__ __forceinline__ C<T> ci(C<T> a) { return {-a.i, a.r}; }    // i a
template <typename T> __device__ __forceinline__ C<T> cmi(C<T> a) { return {a.i, -a.r}; }   // -i a
template <typename T> __device__ __forceinline__ C<T> cneg(C<T> a) { return {-a.r, -a.i}; }
template <typename T> __device__ __forceinline__ C<T> cconj(C<T> a) { return {a.r, -a.i}; }

// ---------------------------------------------------------------- geometry
// Coordinates of site x.  Site indices fit in 32 bits (the lattice volume
// is capped), so the divisions are 32-bit: 64-bit integer division is
// emulated by a long instruction sequence on the GPU.  (Multiply-high
// division here changed the register allocation of the FP32 D for the worse.)
__device__ __forceinline__ void site_coords(const Geom &g, long long x, int c[4])
{
    unsigned r = (unsigned)x;
    const unsigned l0 = (unsigned)g.L[0], l1 = (unsigned)g.L[1], l2 = (unsigned)g.L[2];
    unsigned q = r / l0;
    c[0] = (int)(r - q * l0);
    r = q;
    q = r / l1;
    c[1] = (int)(r - q * l1);
    r = q;
    q = r / l2;
    c[2] = (int)(r - q * l2);
    c[3] = (int)q;
}

__device__ __forceinline__ long long fwd_site(const Geom &g, long long x, const int c[4], int mu)
{
    const unsigned xi = (unsigned)x, st = (unsigned)g.stride[mu];
    return c[mu] == g.L[mu] - 1 ? xi - (unsigned)(g.L[mu] - 1) * st : xi + st;
}

__device__ __forceinline__ long long bwd_site(const Geom &g, long long x, const int c[4], int mu)
{
    const unsigned xi = (unsigned)x, st = (unsigned)g.stride[mu];
    return c[mu] == 0 ? xi + (unsigned)(g.L[mu] - 1) * st : xi - st;
}

// ---------------------------------------------------------------- spinors
// Field planes are indexed in 32 bits: the library caps the volume so that
// the largest field (36 planes of V sites) stays below 2^32 elements, and a
// 32-bit index costs fewer integer instructions per load than a 64-bit one.
template <int P, typename T>
__device__ __forceinline__ void load_spinor(const SpinorView &f, long long V, long long x, C<T> (&s)[12])
{
    const unsigned v = (unsigned)V, i = (unsigned)x;
    if constexpr (P == P64) {
        const double2 *p = (const double2 *)f.d;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            double2 a = p[k * v + i];
            s[k] = {(T)a.x, (T)a.y};
        }
    } else if constexpr (P == P32) {
        const float4 *p = (const float4 *)f.d;
#pragma unroll
        for (int q = 0; q < 6; q++) {
            float4 a = p[q * v + i];
            s[2 * q] = {(T)a.x, (T)a.y};
            s[2 * q + 1] = {(T)a.z, (T)a.w};
        }
    } else {
        const uint4 *p = (const uint4 *)f.d;
        float n = f.n[i];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            uint4 a = p[q * v + i];
            unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                __half2 h = *reinterpret_cast<__half2 *>(&w[j]);
                float2 f2 = __half22float2(h);
                s[4 * q + j] = {(T)(f2.x * n), (T)(f2.y * n)};
            }
        }
    }
}

// As load_spinor, but FP16 values are left unscaled and the site norm is
// returned (1 for FP32/FP64), so that callers fold it into a coefficient.
template <int P, typename T>
__device__ __forceinline__ T load_spinor_u(const SpinorView &f, long long V, long long x, C<T> (&s)[12])
{
    const unsigned v = (unsigned)V, i = (unsigned)x;
    if constexpr (P == P16) {
        const uint4 *p = (const uint4 *)f.d;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            uint4 a = p[q * v + i];
            unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float2 f2 = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
                s[4 * q + j] = {(T)f2.x, (T)f2.y};
            }
        }
        return (T)f.n[i];
    } else {
        load_spinor<P>(f, V, x, s);
        return (T)1;
    }
}

template <int P, typename T>
__device__ __forceinline__ void store_spinor(const SpinorView &f, long long V, long long x, const C<T> (&s)[12])
{
    const unsigned v = (unsigned)V, i = (unsigned)x;
    if constexpr (P == P64) {
        double2 *p = (double2 *)f.d;
#pragma unroll
        for (int k = 0; k < 12; k++) p[k * v + i] = make_double2((double)s[k].r, (double)s[k].i);
    } else if constexpr (P == P32) {
        float4 *p = (float4 *)f.d;
#pragma unroll
        for (int q = 0; q < 6; q++)
            p[q * v + i] = make_float4((float)s[2 * q].r, (float)s[2 * q].i, (float)s[2 * q + 1].r,
                                       (float)s[2 * q + 1].i);
    } else {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf((float)s[k].r), fabsf((float)s[k].i)));
        // a site whose largest component is below 1e-30 is stored as zero: its
        // reciprocal could overflow (FP32 denormals), and such values vanish
        // against the O(1) vectors the solver normalises to
        if (!(m >= 1e-30f)) m = 0.f;
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        uint4 *p = (uint4 *)f.d;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            unsigned w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                __half2 h = __floats2half2_rn((float)s[4 * q + j].r * inv, (float)s[4 * q + j].i * inv);
                w[j] = *reinterpret_cast<unsigned *>(&h);
            }
            p[q * v + i] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        f.n[i] = m;
    }
}

// ---------------------------------------------------------------- links
template <typename T>
__device__ __forceinline__ void rebuild_row2(C<T> (&U)[9])
{
    // row2 = conj(row0 x row1) for an SU(3) matrix
    U[6] = cconj(cfma(U[1], U[5], cneg(cmul(U[2], U[4]))));
    U[7] = cconj(cfma(U[2], U[3], cneg(cmul(U[0], U[5]))));
    U[8] = cconj(cfma(U[0], U[4], cneg(cmul(U[1], U[3]))));
}

template <int P, typename T>
__device__ __forceinline__ void load_link(const LinkView &u, long long V, int mu, long long x, C<T> (&U)[9])
{
    const unsigned v = (unsigned)V, i = (unsigned)x;
    if constexpr (P == P64) {
        const double2 *p = (const double2 *)u.d + mu * 9 * v;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double2 a = p[k * v + i];
            U[k] = {(T)a.x, (T)a.y};
        }
    } else if constexpr (P == P32) {
        const float4 *p = (const float4 *)u.d + mu * 3 * v;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            float4 a = p[q * v + i];
            U[2 * q] = {(T)a.x, (T)a.y};
            U[2 * q + 1] = {(T)a.z, (T)a.w};
        }
        rebuild_row2(U);
    } else {
        const uint2 *p = (const uint2 *)u.d + mu * 3 * v;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            uint2 a = p[q * v + i];
            unsigned w[2] = {a.x, a.y};
#pragma unroll
            for (int j = 0; j < 2; j++) {
                float2 f2 = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
                U[2 * q + j] = {(T)f2.x, (T)f2.y};
            }
        }
        rebuild_row2(U);
    }
}

// ---------------------------------------------------------------- hopping
// acc += c * (1 -+ gamma_mu) (x) M psi, with M = U (forward, minus sign)
// or M = U^dag (backward, plus sign), psi the neighbour's spinor.
template <int MU, bool FWD, typename T>
__device__ __forceinline__ void hop(C<T> (&acc)[12], const C<T> (&s)[12], const C<T> (&U)[9], T c)
{
    C<T> h0[3], h1[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C<T> u0 = s[a], u1 = s[3 + a], d0 = s[6 + a], d1 = s[9 + a];
        C<T> x0, x1;  // X_mu dn
        if constexpr (MU == 0) { x0 = ci(d1); x1 = ci(d0); }
        else if constexpr (MU == 1) { x0 = cneg(d1); x1 = d0; }
        else if constexpr (MU == 2) { x0 = ci(d0); x1 = cmi(d1); }
        else { x0 = d0; x1 = d1; }
        if constexpr (FWD) { h0[a] = csub(u0, x0); h1[a] = csub(u1, x1); }
        else { h0[a] = cadd(u0, x0); h1[a] = cadd(u1, x1); }
    }
    C<T> w0[3], w1[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C<T> p, q;
        if constexpr (FWD) {
            p = cmul(U[a * 3], h0[0]);
            q = cmul(U[a * 3], h1[0]);
        } else {
            p = cmulc(U[a], h0[0]);
            q = cmulc(U[a], h1[0]);
        }
#pragma unroll
        for (int b = 1; b < 3; b++) {
            if constexpr (FWD) {
                p = cfma(U[a * 3 + b], h0[b], p);
                q = cfma(U[a * 3 + b], h1[b], q);
            } else {
                p = cfmac(U[b * 3 + a], h0[b], p);
                q = cfmac(U[b * 3 + a], h1[b], q);
            }
        }
        w0[a] = p;
        w1[a] = q;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        C<T> l0, l1;  // X_mu^dag w
        if constexpr (MU == 0) { l0 = cmi(w1[a]); l1 = cmi(w0[a]); }
        else if constexpr (MU == 1) { l0 = w1[a]; l1 = cneg(w0[a]); }
        else if constexpr (MU == 2) { l0 = cmi(w0[a]); l1 = ci(w1[a]); }
        else { l0 = w0[a]; l1 = w1[a]; }
        if constexpr (FWD) { l0 = cneg(l0); l1 = cneg(l1); }
        acc[a] = cadd(acc[a], cscale(w0[a], c));
        acc[3 + a] = cadd(acc[3 + a], cscale(w1[a], c));
        acc[6 + a] = cadd(acc[6 + a], cscale(l0, c));
        acc[9 + a] = cadd(acc[9 + a], cscale(l1, c));
    }
}

// ---------------------------------------------------------------- clover
template <int P, typename T>
__device__ __forceinline__ void load_clover(const CloverView &A, long long V, long long x, T (&a)[72])
{
    const unsigned v = (unsigned)V, i = (unsigned)x;
    if constexpr (P == P64) {
        const double2 *p = (const double2 *)A.d;
#pragma unroll
        for (int k = 0; k < 36; k++) {
            const double2 e = p[k * v + i];
            a[2 * k] = (T)e.x;
            a[2 * k + 1] = (T)e.y;
        }
    } else if constexpr (P == P32) {
        const float4 *p = (const float4 *)A.d;
#pragma unroll
        for (int k = 0; k < 18; k++) {
            const float4 e = p[k * v + i];
            a[4 * k] = (T)e.x; a[4 * k + 1] = (T)e.y; a[4 * k + 2] = (T)e.z; a[4 * k + 3] = (T)e.w;
        }
    } else {
        // word m of the FP16 clover holds entry m of block 0 (low half) and
        // entry m of block 1 (high half)
        const uint4 *p = (const uint4 *)A.d;
        float n = A.n[i];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const uint4 e = p[k * v + i];
            unsigned w[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float2 f2 = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
                a[4 * k + j] = (T)(f2.x * n);
                a[36 + 4 * k + j] = (T)(f2.y * n);
            }
        }
    }
}

// As load_clover, but FP16 values are left unscaled and the norm returned.
template <int P, typename T>
__device__ __forceinline__ T load_clover_u(const CloverView &A, long long V, long long x, T (&a)[72])
{
    const unsigned v = (unsigned)V, i = (unsigned)x;
    if constexpr (P == P16) {
        const uint4 *p = (const uint4 *)A.d;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const uint4 e = p[k * v + i];
            unsigned w[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float2 f2 = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
                a[4 * k + j] = (T)f2.x;
                a[36 + 4 * k + j] = (T)f2.y;
            }
        }
        return (T)A.n[i];
    } else {
        load_clover<P>(A, V, x, a);
        return (T)1;
    }
}

// Position of the lower off-diagonal element (i > j) of a packed 6x6 block.
__host__ __device__ constexpr int cl_off(int i, int j) { return 6 + 2 * (i * (i - 1) / 2 + j); }

// out = A psi with A the two packed Hermitian 6x6 chiral blocks.
template <typename T>
__device__ __forceinline__ void clover_apply(const T (&a)[72], const C<T> (&s)[12], C<T> (&o)[12])
{
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int base = 36 * h;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            C<T> acc = cscale(s[6 * h + i], a[base + i]);
#pragma unroll
            for (int j = 0; j < 6; j++) {
                if (j < i) {
                    C<T> l = {a[base + cl_off(i, j)], a[base + cl_off(i, j) + 1]};
                    acc = cfma(l, s[6 * h + j], acc);
                } else if (j > i) {
                    C<T> l = {a[base + cl_off(j, i)], a[base + cl_off(j, i) + 1]};
                    acc = cfmac(l, s[6 * h + j], acc);
                }
            }
            o[6 * h + i] = acc;
        }
    }
}

// ---------------------------------------------------------------- D at one site
// (D in)(x) = A(x) in(x) - kappa sum_mu [hops], all fields read from global
// memory in the precision P; FP16 norms are folded into the coefficients.
template <int P, int MU, typename T>
__device__ __forceinline__ void hop_pair(const Geom &g, const SpinorView &in, const LinkView &Ul, long long x,
                                         const int c[4], C<T> (&acc)[12], T mk)
{
    const long long V = g.V;
    {
        const long long xf = fwd_site(g, x, c, MU);
        const T sf = (c[MU] == g.L[MU] - 1 && g.bc[MU] < 0) ? -mk : mk;
        C<T> s[12], U[9];
        const T nf = load_spinor_u<P>(in, V, xf, s);
        load_link<P>(Ul, V, MU, x, U);
        hop<MU, true>(acc, s, U, sf * nf);
    }
    {
        const long long xb = bwd_site(g, x, c, MU);
        const T sb = (c[MU] == 0 && g.bc[MU] < 0) ? -mk : mk;
        C<T> s[12], U[9];
        const T nb = load_spinor_u<P>(in, V, xb, s);
        load_link<P>(Ul, V, MU, xb, U);
        hop<MU, false>(acc, s, U, sb * nb);
    }
}

// Clover block H (0: spins 0,1; 1: spins 2,3) of the packed site clover,
// the 36 reals [36 H, 36 H + 36): 6 diagonal reals, then the 15 complex
// lower entries.  FP16 values are left unscaled (the site norm is applied by
// the caller).
template <int P, int H, typename T>
__device__ __forceinline__ void load_clover_block(const CloverView &A, long long V, long long x, T (&a)[36])
{
    const unsigned v = (unsigned)V, i = (unsigned)x;
    if constexpr (P == P64) {
        const double2 *p = (const double2 *)A.d;
#pragma unroll
        for (int k = 0; k < 18; k++) {
            const double2 e = p[(18 * H + k) * v + i];
            a[2 * k] = (T)e.x;
            a[2 * k + 1] = (T)e.y;
        }
    } else if constexpr (P == P32) {
        const float4 *p = (const float4 *)A.d;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const float4 e = p[(9 * H + k) * v + i];
            a[4 * k] = (T)e.x; a[4 * k + 1] = (T)e.y; a[4 * k + 2] = (T)e.z; a[4 * k + 3] = (T)e.w;
        }
    } else {
        // block H is the low (H = 0) or high (H = 1) half of every word
        const uint4 *p = (const uint4 *)A.d;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const uint4 e = p[k * v + i];
            unsigned w[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float2 f2 = __half22float2(*reinterpret_cast<__half2 *>(&w[j]));
                a[4 * k + j] = (T)(H == 0 ? f2.x : f2.y);
            }
        }
    }
}

// o += sc * B s for one packed Hermitian 6x6 block B.
template <typename T>
__device__ __forceinline__ void clover_block_acc(const T (&a)[36], const C<T> *s, C<T> *o, T sc)
{
#pragma unroll
    for (int i = 0; i < 6; i++) {
        C<T> t = cscale(s[i], a[i]);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            if (j < i) t = cfma(C<T>{a[cl_off(i, j)], a[cl_off(i, j) + 1]}, s[j], t);
            else if (j > i) t = cfmac(C<T>{a[cl_off(j, i)], a[cl_off(j, i) + 1]}, s[j], t);
        }
        o[i].r = fma(sc, t.r, o[i].r);
        o[i].i = fma(sc, t.i, o[i].i);
    }
}

// D at site x.  FP32/FP64: clover term first, then the hops.  FP16: the hops
// first, then the clover block by block, so that the clover's 72 reals are
// never live together with the hop temporaries (the FP16 kernels are bounded
// to 80 registers for occupancy).
template <int P, typename T>
__device__ __forceinline__ void apply_D_site(const Geom &g, const SpinorView &in, const LinkView &Ul,
                                             const CloverView &A, T kappa, long long x, C<T> (&acc)[12])
{
    const long long V = g.V;
    int c[4];
    site_coords(g, x, c);
    const T mk = -kappa;
    if constexpr (P == P16) {
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = {0, 0};
        hop_pair<P, 0>(g, in, Ul, x, c, acc, mk);
        hop_pair<P, 1>(g, in, Ul, x, c, acc, mk);
        hop_pair<P, 2>(g, in, Ul, x, c, acc, mk);
        hop_pair<P, 3>(g, in, Ul, x, c, acc, mk);
        C<T> s[12];
        const T sc = load_spinor_u<P>(in, V, x, s) * (T)A.n[(unsigned)x];
        {
            T ab[36];
            load_clover_block<P, 0>(A, V, x, ab);
            clover_block_acc(ab, s, acc, sc);
        }
        {
            T ab[36];
            load_clover_block<P, 1>(A, V, x, ab);
            clover_block_acc(ab, s + 6, acc + 6, sc);
        }
    } else {
        {
            T av[72];
            C<T> s[12];
            load_clover<P>(A, V, x, av);
            load_spinor<P>(in, V, x, s);
            clover_apply(av, s, acc);
        }
        hop_pair<P, 0>(g, in, Ul, x, c, acc, mk);
        hop_pair<P, 1>(g, in, Ul, x, c, acc, mk);
        hop_pair<P, 2>(g, in, Ul, x, c, acc, mk);
        hop_pair<P, 3>(g, in, Ul, x, c, acc, mk);
    }
}

// ---------------------------------------------------------------- reductions
// Sum over the block of one value per thread and component; the total ends
// up in v in every lane of warp 0 (thread 0 in particular).  The warp stage
// runs in the callers' type T: FP32 in the FP32/FP16 kernels, whose per-site
// terms are FP32 already, because FP64 adds and conversions run at a small
// fraction of the FP32 rate on this GPU and would otherwise cost more than
// the site arithmetic of a bandwidth-bound kernel.  The warp totals are added
// in FP64.  in and v may be the same array.  All threads must call it.
template <int N, typename T>
__device__ __forceinline__ void block_sum(T (&in)[N], double (&v)[N], double *sm /* N * 32 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) in[k] += __shfl_xor_sync(0xffffffffu, in[k], o);
    __syncthreads();  // sm may be in use by a previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; k++) sm[k * 32 + warp] = (double)in[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; k++) {
            v[k] = lane < nw ? sm[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        }
    }
}

template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double *sm /* N * 32 */)
{
    block_sum<N, double>(v, v, sm);
}

// Block sum that leaves the total in every thread of the block.
template <int N>
__device__ __forceinline__ void block_allsum(double (&v)[N], double *sm /* N * 32 + N */)
{
    block_sum<N>(v, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < N; k++) sm[N * 32 + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; k++) v[k] = sm[N * 32 + k];
}

// Grid-wide sum by the last-block pattern over the nblk blocks that share
// one reduction (one right-hand side): every block stores its partial sums,
// and the block that arrives last adds them in block order (so the result
// does not depend on scheduling) and returns true in thread 0 with the
// totals in v.  No block waits for another.  The per-thread values t are of
// the kernel's type T (see block_sum).
template <int N, typename T>
__device__ __forceinline__ bool grid_sum(T (&t)[N], double (&v)[N], double *partials, unsigned int *counter,
                                         unsigned bid, unsigned nblk)
{
    __shared__ double sm[N * 32];
    __shared__ int last;
    block_sum<N, T>(t, v, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; k++) partials[(long long)bid * N + k] = v[k];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[N];
#pragma unroll
    for (int k = 0; k < N; k++) acc[k] = 0.0;
    // unrolled so that several L2 loads are in flight per thread: this block
    // runs alone at the end of the kernel, so its latency is the kernel's tail
#pragma unroll 8
    for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < N; k++) acc[k] += __ldcg(partials + (long long)b * N + k);
    block_sum<N>(acc, sm);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; k++) v[k] = acc[k];
        *counter = 0u;
    }
    return threadIdx.x == 0;
}

// The lattice of this block in a work-list launch, whose lattice i owns the
// blocks first[i] .. first[i+1]-1 (n lattices).
__device__ __forceinline__ int list_member(const int *first, int n)
{
    int i = 0;
    while (i + 1 < n && (int)blockIdx.x >= first[i + 1]) i++;
    return i;
}

// dst = src (bytes a multiple of 4), by all threads of the block.
__device__ __forceinline__ void copy_words(void *dst, const void *src, unsigned bytes)
{
    for (unsigned k = threadIdx.x; k < bytes / 4; k += blockDim.x)
        static_cast<unsigned *>(dst)[k] = static_cast<const unsigned *>(src)[k];
}

// Reduction scratch of right-hand side r.
__device__ __forceinline__ double *rs_partials(const ReduceScratch &rs, int r)
{
    return rs.partials + (long long)r * rs.max_blocks * 4;
}
__device__ __forceinline__ unsigned int *rs_counter(const ReduceScratch &rs, int r) { return rs.counter + r * 16; }

// The field of right-hand side r inside a multi-RHS field (R vectors stored
// one after the other, each in the planar layout of its precision).
template <int P>
__device__ __forceinline__ SpinorView rhs_view(SpinorView f, long long V, int r)
{
    if (!f.d) return f;
    if constexpr (P == P64) f.d = (double2 *)f.d + (long long)r * 12 * V;
    else if constexpr (P == P32) f.d = (float4 *)f.d + (long long)r * 6 * V;
    else {
        f.d = (uint4 *)f.d + (long long)r * 3 * V;
        f.n = f.n + (long long)r * V;
    }
    return f;
}

// ---------------------------------------------------------------- scalars
__device__ __forceinline__ double2 zdiv(double2 a, double2 b)
{
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

}  // namespace qdd
