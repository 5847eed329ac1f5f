// lattice.cu -- layout conversions, gauge-field import and the clover term.
//
// The clover term is the O(a) improvement of the Wilson quark named in
// Sec. 1 and Sec. 5 (coefficient c_SW):
//     A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x),
//     Fhat_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dag) / 8,
// Q the sum of the four plaquette leaves at x in the (mu, nu) plane.  In the
// DeGrand-Rossi basis sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] is block
// diagonal in chirality; writing its 2x2 blocks with Pauli matrices
// (s_x, s_y, s_z) gives, for the upper (spins 0,1) and lower (spins 2,3)
// blocks,
//     upper: s_z (F_xy - F_zt) + s_y (F_xz + F_yt) + s_x (F_yz - F_xt)
//     lower: s_z (F_xy + F_zt) + s_y (F_xz - F_yt) + s_x (F_yz + F_xt)
// so each 6x6 block is 1 + i kappa c_sw [[Gz, Gx - i Gy], [Gx + i Gy, -Gz]].
// The build runs once per (gauge field, kappa, c_sw) in FP64 and stores the
// result in all three working precisions.
#include "device.cuh"
#include "df64.cuh"
#include "lib.h"

namespace qdd {

// ---------------------------------------------------------------- spinors
template <int P>
__global__ void import_spinor_kernel(Geom g, SpinorView dst, const double *src)
{
    typedef typename RealOf<P>::T T;
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    dst = rhs_view<P>(dst, g.V, blockIdx.y);
    const double2 *s2 = reinterpret_cast<const double2 *>(src) + ((long long)blockIdx.y * g.V + x) * 12;
    C<T> s[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
        double2 v = s2[k];
        s[k] = {(T)v.x, (T)v.y};
    }
    store_spinor<P>(dst, g.V, x, s);
}

template <int P>
__global__ void export_spinor_kernel(Geom g, double *dst, SpinorView src)
{
    typedef typename RealOf<P>::T T;
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    src = rhs_view<P>(src, g.V, blockIdx.y);
    C<T> s[12];
    load_spinor<P>(src, g.V, x, s);
    double2 *d2 = reinterpret_cast<double2 *>(dst) + ((long long)blockIdx.y * g.V + x) * 12;
#pragma unroll
    for (int k = 0; k < 12; k++) d2[k] = make_double2((double)s[k].r, (double)s[k].i);
}

cudaError_t launch_import_spinor(const Geom &g, int prec, SpinorView dst, const double *src, int nrhs,
                                 cudaStream_t st)
{
    const dim3 nb((unsigned)((g.V + 255) / 256), (unsigned)nrhs);
    if (prec == P64) import_spinor_kernel<P64><<<nb, 256, 0, st>>>(g, dst, src);
    else if (prec == P32) import_spinor_kernel<P32><<<nb, 256, 0, st>>>(g, dst, src);
    else import_spinor_kernel<P16><<<nb, 256, 0, st>>>(g, dst, src);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_export_spinor(const Geom &g, int prec, double *dst, SpinorView src, int nrhs, cudaStream_t st)
{
    const dim3 nb((unsigned)((g.V + 255) / 256), (unsigned)nrhs);
    if (prec == P64) export_spinor_kernel<P64><<<nb, 256, 0, st>>>(g, dst, src);
    else if (prec == P32) export_spinor_kernel<P32><<<nb, 256, 0, st>>>(g, dst, src);
    else export_spinor_kernel<P16><<<nb, 256, 0, st>>>(g, dst, src);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gauge
__global__ void gauge_convert_kernel(Geom g, const double *U, double2 *U64, float4 *U32, uint2 *U16, float4 *Udf,
                                     unsigned long long *maxdev)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double dev = 0.0;
    if (t < g.V * 4) {
        const long long x = t >> 2;
        const int mu = (int)(t & 3);
        const double2 *u2 = reinterpret_cast<const double2 *>(U) + t * 9;
        C<double> m[9];
        CDF d[9];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double2 v = u2[k];
            m[k] = {v.x, v.y};
            d[k] = CDF{df_from_double(v.x), df_from_double(v.y)};
        }
        // SU(3) check in double-float: max |(U^dag U - 1)_{ab}| and |det U - 1|
        const CDF z = CDF{DF{0.f, 0.f}, DF{0.f, 0.f}};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                CDF s = z;
                if (a == b) s.r = DF{-1.f, 0.f};
#pragma unroll
                for (int k = 0; k < 3; k++) s = cdf_fma_ca(d[k * 3 + a], d[k * 3 + b], s);
                const double re = df_to_double(s.r), im = df_to_double(s.i);
                dev = fmax(dev, sqrt(re * re + im * im));
            }
        {
            // det = u00 (u11 u22 - u12 u21) - u01 (u10 u22 - u12 u20) + u02 (u10 u21 - u11 u20)
            auto minor = [&](int a, int b, int c, int e) {  // d[a] d[b] - d[c] d[e]
                CDF t = cdf_fma(d[a], d[b], z);
                CDF mc = CDF{df_neg(d[c].r), df_neg(d[c].i)};
                return cdf_fma(mc, d[e], t);
            };
            CDF det = cdf_fma(d[0], minor(4, 8, 5, 7), z);
            const CDF m1 = minor(3, 8, 5, 6);
            det = cdf_fma(CDF{df_neg(d[1].r), df_neg(d[1].i)}, m1, det);
            det = cdf_fma(d[2], minor(3, 7, 4, 6), det);
            const double re = df_to_double(df_add(det.r, DF{-1.f, 0.f})), im = df_to_double(det.i);
            dev = fmax(dev, sqrt(re * re + im * im));
        }
        if (!isfinite(dev)) dev = 1e300;

        const long long V = g.V;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            U64[((long long)mu * 9 + k) * V + x] = make_double2(m[k].r, m[k].i);
            Udf[((long long)mu * 9 + k) * V + x] = make_float4(d[k].r.h, d[k].r.l, d[k].i.h, d[k].i.l);
        }
#pragma unroll
        for (int q = 0; q < 3; q++) {
            U32[((long long)mu * 3 + q) * V + x] =
                make_float4((float)m[2 * q].r, (float)m[2 * q].i, (float)m[2 * q + 1].r, (float)m[2 * q + 1].i);
            __half2 h0 = __floats2half2_rn((float)m[2 * q].r, (float)m[2 * q].i);
            __half2 h1 = __floats2half2_rn((float)m[2 * q + 1].r, (float)m[2 * q + 1].i);
            U16[((long long)mu * 3 + q) * V + x] =
                make_uint2(*reinterpret_cast<unsigned *>(&h0), *reinterpret_cast<unsigned *>(&h1));
        }
    }
    // block max, then one atomic per block on the bit pattern (non-negative
    // doubles order like their bit patterns)
    for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxdev, (unsigned long long)__double_as_longlong(dev));
}

cudaError_t launch_gauge_convert(const Geom &g, const double *U, void *U64, void *U32, void *U16, void *Udf,
                                 unsigned long long *maxdev, cudaStream_t st)
{
    const long long n = g.V * 4;
    const unsigned nb = (unsigned)((n + 255) / 256);
    gauge_convert_kernel<<<nb, 256, 0, st>>>(g, U, (double2 *)U64, (float4 *)U32, (uint2 *)U16, (float4 *)Udf,
                                             maxdev);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- clover
typedef C<double> Z;

// 3x3 complex matrices in double-float arithmetic (df64.cuh).
struct M3D {
    CDF e[9];
};

__device__ __forceinline__ M3D md_load(const float4 *Udf, long long V, int mu, long long x)
{
    M3D m;
    const float4 *p = Udf + (long long)mu * 9 * V;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const float4 v = p[k * V + x];
        m.e[k] = CDF{DF{v.x, v.y}, DF{v.z, v.w}};
    }
    return m;
}

__device__ __forceinline__ M3D md_zero()
{
    M3D c;
#pragma unroll
    for (int k = 0; k < 9; k++) c.e[k] = CDF{DF{0.f, 0.f}, DF{0.f, 0.f}};
    return c;
}

__device__ __forceinline__ M3D md_mul(const M3D &a, const M3D &b)  // a b
{
    M3D c = md_zero();
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int k = 0; k < 3; k++) c.e[i * 3 + j] = cdf_fma(a.e[i * 3 + k], b.e[k * 3 + j], c.e[i * 3 + j]);
    return c;
}

__device__ __forceinline__ M3D md_mul_d(const M3D &a, const M3D &b)  // a b^dag
{
    M3D c = md_zero();
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int k = 0; k < 3; k++) c.e[i * 3 + j] = cdf_fma_cb(a.e[i * 3 + k], b.e[j * 3 + k], c.e[i * 3 + j]);
    return c;
}

__device__ __forceinline__ M3D md_dmul(const M3D &a, const M3D &b)  // a^dag b
{
    M3D c = md_zero();
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int k = 0; k < 3; k++) c.e[i * 3 + j] = cdf_fma_ca(a.e[k * 3 + i], b.e[k * 3 + j], c.e[i * 3 + j]);
    return c;
}

__device__ __forceinline__ M3D md_dag(const M3D &a)
{
    M3D c;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) c.e[i * 3 + j] = CDF{a.e[j * 3 + i].r, df_neg(a.e[j * 3 + i].i)};
    return c;
}

__device__ __forceinline__ void md_acc(M3D &q, const M3D &l)
{
#pragma unroll
    for (int k = 0; k < 9; k++) q.e[k] = CDF{df_add(q.e[k].r, l.e[k].r), df_add(q.e[k].i, l.e[k].i)};
}

__device__ __forceinline__ long long shifted(const Geom &g, const int c[4], int mu, int dm, int nu, int dn)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + dm + g.L[mu]) % g.L[mu];
    d[nu] = (d[nu] + dn + g.L[nu]) % g.L[nu];
    return d[0] + g.stride[1] * d[1] + g.stride[2] * d[2] + g.stride[3] * d[3];
}

// Fhat_{mu nu}(x) = (Q - Q^dag) / 8 from the four counter-clockwise leaves,
// in double-float arithmetic; returned as FP64 (18 reals, row-major re/im).
__device__ void field_strength(const Geom &g, const float4 *Udf, long long x, const int c[4], int mu, int nu,
                               double (&F)[18])
{
    const long long V = g.V;
    const long long xpm = shifted(g, c, mu, 1, nu, 0), xpn = shifted(g, c, mu, 0, nu, 1);
    const long long xmm = shifted(g, c, mu, -1, nu, 0), xmn = shifted(g, c, mu, 0, nu, -1);
    const long long xmm_pn = shifted(g, c, mu, -1, nu, 1), xmm_mn = shifted(g, c, mu, -1, nu, -1);
    const long long xpm_mn = shifted(g, c, mu, 1, nu, -1);
    // x -> x+mu -> x+mu+nu -> x+nu -> x
    M3D Q = md_mul(md_load(Udf, V, mu, x), md_load(Udf, V, nu, xpm));
    Q = md_mul_d(Q, md_load(Udf, V, mu, xpn));
    Q = md_mul_d(Q, md_load(Udf, V, nu, x));
    // x -> x+nu -> x-mu+nu -> x-mu -> x
    M3D l = md_mul_d(md_load(Udf, V, nu, x), md_load(Udf, V, mu, xmm_pn));
    l = md_mul_d(l, md_load(Udf, V, nu, xmm));
    l = md_mul(l, md_load(Udf, V, mu, xmm));
    md_acc(Q, l);
    // x -> x-mu -> x-mu-nu -> x-nu -> x:  U_mu(x-mu)^dag U_nu(x-mu-nu)^dag = (U_nu(x-mu-nu) U_mu(x-mu))^dag
    l = md_dag(md_mul(md_load(Udf, V, nu, xmm_mn), md_load(Udf, V, mu, xmm)));
    l = md_mul(l, md_load(Udf, V, mu, xmm_mn));
    l = md_mul(l, md_load(Udf, V, nu, xmn));
    md_acc(Q, l);
    // x -> x-nu -> x+mu-nu -> x+mu -> x
    l = md_dmul(md_load(Udf, V, nu, xmn), md_load(Udf, V, mu, xmn));
    l = md_mul(l, md_load(Udf, V, nu, xpm_mn));
    l = md_mul_d(l, md_load(Udf, V, mu, x));
    md_acc(Q, l);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const CDF q = Q.e[i * 3 + j], qt = Q.e[j * 3 + i];
            // (Q - Q^dag)_{ij} / 8 = (q - conj(qt)) / 8
            F[2 * (i * 3 + j)] = df_to_double(df_scale2(df_sub(q.r, qt.r), 0.125f));
            F[2 * (i * 3 + j) + 1] = df_to_double(df_scale2(df_add(q.i, qt.i), 0.125f));
        }
}

// One CTA builds the clover of 32 consecutive sites in three phases:
//  1. warp p (p = 0..5, the planes xy xz xt yz yt zt) computes Fhat_p of its
//     site (lane) and leaves it in shared memory;
//  2. 64 threads (site, chirality h) pack the Hermitian 6x6 block h from the
//     six Fhat's (36 reals);
//  3. 32 threads store each site in FP64, FP32 and FP16 (with its norm).
// Holding one Fhat per thread instead of six keeps the FP64 leaf products
// in registers.
constexpr int CL_SITES = 32;

__global__ void __launch_bounds__(6 * CL_SITES, 2) clover_build_kernel(Geom g, const float4 *Udf, double kappa,
                                                                     double csw, double2 *A64, float4 *A32,
                                                                     uint4 *A16, float *A16n)
{
    __shared__ double sF[6][18][CL_SITES];
    __shared__ double sP[72][CL_SITES];
    const int lane = threadIdx.x % CL_SITES;
    const long long x = (long long)blockIdx.x * CL_SITES + lane;
    const bool act = x < g.V;
    {
        const int plane = threadIdx.x / CL_SITES;
        // planes (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
        const int mu = (plane >= 3) + (plane >= 5);
        const int nu = plane < 3 ? plane + 1 : plane < 5 ? plane - 1 : 3;
        if (act) {
            int c[4];
            site_coords(g, x, c);
            double F[18];
            field_strength(g, Udf, x, c, mu, nu, F);
#pragma unroll
            for (int k = 0; k < 18; k++) sF[plane][k][lane] = F[k];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * CL_SITES && act) {
        // block h: 1 + i kc [[Gz, Gx - i Gy], [Gx + i Gy, -Gz]] with
        //   Gz = F_xy -+ F_zt, Gy = F_xz +- F_yt, Gx = F_yz -+ F_xt (upper / lower)
        const int h = threadIdx.x / CL_SITES;
        const double sg = h == 0 ? -1.0 : 1.0;
        const double kc = kappa * csw;
        auto G = [&](int which, int a, int b) -> Z {
            const int k = a * 3 + b;
            int p0, p1;
            double w;
            if (which == 0) { p0 = 0; p1 = 5; w = sg; }          // Gz = F_xy + sg F_zt
            else if (which == 1) { p0 = 1; p1 = 4; w = -sg; }    // Gy = F_xz - sg F_yt
            else { p0 = 3; p1 = 2; w = sg; }                     // Gx = F_yz + sg F_xt
            return Z{sF[p0][2 * k][lane] + w * sF[p1][2 * k][lane], sF[p0][2 * k + 1][lane] + w * sF[p1][2 * k + 1][lane]};
        };
        auto M = [&](int i, int j) -> Z {
            const int s = i / 3, a = i % 3, t = j / 3, b = j % 3;
            Z bst;
            if (s == 0 && t == 0) bst = G(0, a, b);
            else if (s == 1 && t == 1) bst = cneg(G(0, a, b));
            else if (s == 0) bst = csub(G(2, a, b), ci(G(1, a, b)));
            else bst = cadd(G(2, a, b), ci(G(1, a, b)));
            Z m = cscale(ci(bst), kc);
            if (i == j) m.r += 1.0;
            return m;
        };
        const int base = 36 * h;
#pragma unroll 1
        for (int i = 0; i < 6; i++) sP[base + i][lane] = M(i, i).r;
#pragma unroll 1
        for (int i = 1; i < 6; i++)
#pragma unroll 1
            for (int j = 0; j < i; j++) {
                const Z m = M(i, j);
                sP[base + cl_off(i, j)][lane] = m.r;
                sP[base + cl_off(i, j) + 1][lane] = m.i;
            }
    }
    __syncthreads();
    if (threadIdx.x < CL_SITES && act) {
        const long long V = g.V;
        double nrm = 0.0;
#pragma unroll 1
        for (int k = 0; k < 72; k++) nrm = fmax(nrm, fabs(sP[k][lane]));
        const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
#pragma unroll 1
        for (int k = 0; k < 36; k++) A64[k * V + x] = make_double2(sP[2 * k][lane], sP[2 * k + 1][lane]);
#pragma unroll 1
        for (int k = 0; k < 18; k++)
            A32[k * V + x] = make_float4((float)sP[4 * k][lane], (float)sP[4 * k + 1][lane], (float)sP[4 * k + 2][lane],
                                         (float)sP[4 * k + 3][lane]);
#pragma unroll 1
        for (int k = 0; k < 9; k++) {
            unsigned w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                __half2 hh = __floats2half2_rn((float)(sP[8 * k + 2 * j][lane] * inv),
                                               (float)(sP[8 * k + 2 * j + 1][lane] * inv));
                w[j] = *reinterpret_cast<unsigned *>(&hh);
            }
            A16[k * V + x] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        A16n[x] = (float)nrm;
    }
}

cudaError_t launch_clover_build(const Geom &g, const void *Udf, double kappa, double csw, void *A64, void *A32,
                                void *A16, float *A16n, cudaStream_t st)
{
    const unsigned nb = (unsigned)((g.V + CL_SITES - 1) / CL_SITES);
    clover_build_kernel<<<nb, 6 * CL_SITES, 0, st>>>(g, (const float4 *)Udf, kappa, csw, (double2 *)A64, (float4 *)A32,
                                            (uint4 *)A16, A16n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace qdd
