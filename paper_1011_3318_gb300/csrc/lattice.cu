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
// max(a, b) where a NaN b counts as the largest deviation (fmaxf would drop it)
__device__ __forceinline__ float dev_max(float a, float b) { return (b <= 3.0e38f) ? fmaxf(a, b) : 3.0e38f; }

// One block converts the 4 links of GC_SITES consecutive sites.  The
// canonical links of those sites are one contiguous range of 144-byte
// records: the block reads it with coalesced 16-byte loads into shared
// memory, and thread (mu, site) takes its record from there, so that a warp
// then writes 32 consecutive sites of one plane of each internal copy.
constexpr int GC_SITES = 64;
constexpr int GC_THREADS = 4 * GC_SITES;

__global__ void __launch_bounds__(GC_THREADS) gauge_convert_kernel(Geom g, const double *U, double2 *U64, float4 *U32,
                                                                  uint2 *U16, float4 *Udf, unsigned long long *maxdev,
                                                                  long long site0, long long site1)
{
    // a site's 36 complex numbers at a stride of 37 (16-byte units), so that
    // the 32 sites a warp reads fall into different shared-memory banks
    constexpr int SREC = 37;
    __shared__ double2 srec[GC_SITES * SREC];
    const long long xb = site0 + (long long)blockIdx.x * GC_SITES;  // first site of the block
    const long long nsite = min((long long)GC_SITES, site1 - xb);
    {
        const double2 *src = reinterpret_cast<const double2 *>(U) + xb * 36;
        const int n = (int)nsite * 36;
        for (int i = threadIdx.x; i < n; i += GC_THREADS) srec[(i / 36) * SREC + i % 36] = src[i];
    }
    __syncthreads();
    const int mu = threadIdx.x / GC_SITES, ls = threadIdx.x % GC_SITES;
    const long long x = xb + ls;
    float dev = 0.f;
    if (ls < nsite) {
        const double2 *u2 = srec + ls * SREC + mu * 9;
        C<double> m[9];
        CDF d[9];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double2 v = u2[k];
            m[k] = {v.x, v.y};
            d[k] = CDF{df_from_double_i(v.x), df_from_double_i(v.y)};
        }
        // SU(3) check in double-float: max |(U^dag U - 1)_{ab}| and |det U - 1|.
        // The deviations are formed in double-float; their high words carry
        // them to ~1e-22 absolute, so the magnitudes are taken in FP32.
        float devf = 0.f;
        const CDF z = CDF{DF{0.f, 0.f}, DF{0.f, 0.f}};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                CDF s = z;
                if (a == b) s.r = DF{-1.f, 0.f};
#pragma unroll
                for (int k = 0; k < 3; k++) s = cdf_fma_ca(d[k * 3 + a], d[k * 3 + b], s);
                devf = dev_max(devf, sqrtf(s.r.h * s.r.h + s.i.h * s.i.h));
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
            const DF dr = df_add(det.r, DF{-1.f, 0.f});
            devf = dev_max(devf, sqrtf(dr.h * dr.h + det.i.h * det.i.h));
        }
        dev = isfinite(devf) ? devf : 3.0e38f;

        const long long V = g.V;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            U64[((long long)mu * 9 + k) * V + x] = make_double2(m[k].r, m[k].i);
            Udf[((long long)mu * 9 + k) * V + x] = make_float4(d[k].r.h, d[k].r.l, d[k].i.h, d[k].i.l);
        }
#pragma unroll
        for (int q = 0; q < 3; q++) {
            // float(u) is the double-float high word
            U32[((long long)mu * 3 + q) * V + x] =
                make_float4(d[2 * q].r.h, d[2 * q].i.h, d[2 * q + 1].r.h, d[2 * q + 1].i.h);
            __half2 h0 = __floats2half2_rn(d[2 * q].r.h, d[2 * q].i.h);
            __half2 h1 = __floats2half2_rn(d[2 * q + 1].r.h, d[2 * q + 1].i.h);
            U16[((long long)mu * 3 + q) * V + x] =
                make_uint2(*reinterpret_cast<unsigned *>(&h0), *reinterpret_cast<unsigned *>(&h1));
        }
    }
    // warp max in FP32, then one atomic per warp on the bit pattern of the
    // double (non-negative doubles order like their bit patterns)
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(maxdev, (unsigned long long)__double_as_longlong(dev >= 3.0e38f ? 1e300 : (double)dev));
}

cudaError_t launch_gauge_convert(const Geom &g, const double *U, void *U64, void *U32, void *U16, void *Udf,
                                 unsigned long long *maxdev, cudaStream_t st, long long site0, long long site1)
{
    if (site1 < 0) site1 = g.V;
    const long long n = site1 - site0;
    if (n <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((n + GC_SITES - 1) / GC_SITES);
    gauge_convert_kernel<<<nb, GC_THREADS, 0, st>>>(g, U, (double2 *)U64, (float4 *)U32, (uint2 *)U16, (float4 *)Udf,
                                                    maxdev, site0, site1);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- clover
typedef C<double> Z;

__device__ __forceinline__ long long shifted(const Geom &g, const int c[4], int mu, int dm, int nu, int dn)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    // dm, dn in {-1, 0, 1}: one conditional wrap each
    d[mu] += dm;
    d[mu] += d[mu] < 0 ? g.L[mu] : (d[mu] >= g.L[mu] ? -g.L[mu] : 0);
    d[nu] += dn;
    d[nu] += d[nu] < 0 ? g.L[nu] : (d[nu] >= g.L[nu] ? -g.L[nu] : 0);
    return d[0] + g.stride[1] * d[1] + g.stride[2] * d[2] + g.stride[3] * d[3];
}

// A link factor of a plaquette leaf, M = U_mu(y) or U_mu(y)^dag, as an
// element accessor: M_ab is the double-float element at Udf[off + a sa + b sb]
// with its imaginary part multiplied by sg (the dagger swaps the strides and
// conjugates).  Offsets are 32-bit (the volume cap keeps 36 V below 2^32).
struct LinkFactor {
    unsigned off, sa, sb;
    float sg;
};

__device__ __forceinline__ LinkFactor link_factor(unsigned V, int mu, long long y, bool dag)
{
    LinkFactor f;
    f.off = (unsigned)(mu * 9) * V + (unsigned)y;
    f.sa = dag ? V : 3 * V;
    f.sb = dag ? 3 * V : V;
    f.sg = dag ? -1.f : 1.f;
    return f;
}

__device__ __forceinline__ CDF lf_elem(const float4 *Udf, const LinkFactor &f, int a, int b)
{
    const float4 e = Udf[f.off + a * f.sa + b * f.sb];
    return CDF{DF{e.x, e.y}, DF{e.z * f.sg, e.w * f.sg}};
}

// v <- M v in double-float: each output component is two real dot products
// of length 6, summed with DFAcc.
__device__ __forceinline__ void md_apply(const float4 *Udf, const LinkFactor &f, CDF (&v)[3])
{
    CDF w[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        DFAcc re, im;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const CDF u = lf_elem(Udf, f, a, b);
            if (b == 0) {
                dfacc_init(re, u.r, v[b].r);
                dfacc_init(im, u.r, v[b].i);
            } else {
                dfacc_add(re, u.r, v[b].r);
                dfacc_add(im, u.r, v[b].i);
            }
            dfacc_add(re, df_neg(u.i), v[b].i);
            dfacc_add(im, u.i, v[b].r);
        }
        w[a] = CDF{dfacc_result(re), dfacc_result(im)};
    }
#pragma unroll
    for (int a = 0; a < 3; a++) v[a] = w[a];
}

// The four counter-clockwise plaquette leaves at x in the (mu, nu) plane,
// each a product F0 F1 F2 F3 of links: site, direction and dagger of each.
__device__ __forceinline__ void leaf_factors(const Geom &g, const int c[4], long long x, int mu, int nu, int leaf,
                                             long long fx[4], int fd[4], bool fdag[4])
{
    if (leaf == 0) {  // U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
        fx[0] = x;                             fd[0] = mu; fdag[0] = false;
        fx[1] = shifted(g, c, mu, 1, nu, 0);   fd[1] = nu; fdag[1] = false;
        fx[2] = shifted(g, c, mu, 0, nu, 1);   fd[2] = mu; fdag[2] = true;
        fx[3] = x;                             fd[3] = nu; fdag[3] = true;
    } else if (leaf == 1) {  // U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
        fx[0] = x;                             fd[0] = nu; fdag[0] = false;
        fx[1] = shifted(g, c, mu, -1, nu, 1);  fd[1] = mu; fdag[1] = true;
        fx[2] = shifted(g, c, mu, -1, nu, 0);  fd[2] = nu; fdag[2] = true;
        fx[3] = fx[2];                         fd[3] = mu; fdag[3] = false;
    } else if (leaf == 2) {  // U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
        fx[0] = shifted(g, c, mu, -1, nu, 0);  fd[0] = mu; fdag[0] = true;
        fx[1] = shifted(g, c, mu, -1, nu, -1); fd[1] = nu; fdag[1] = true;
        fx[2] = fx[1];                         fd[2] = mu; fdag[2] = false;
        fx[3] = shifted(g, c, mu, 0, nu, -1);  fd[3] = nu; fdag[3] = false;
    } else {  // U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
        fx[0] = shifted(g, c, mu, 0, nu, -1);  fd[0] = nu; fdag[0] = true;
        fx[1] = fx[0];                         fd[1] = mu; fdag[1] = false;
        fx[2] = shifted(g, c, mu, 1, nu, -1);  fd[2] = nu; fdag[2] = false;
        fx[3] = x;                             fd[3] = mu; fdag[3] = true;
    }
}

// One CTA builds the clover of CL_SITES consecutive sites in three phases:
//  1. thread (plane, site) forms Q = sum of the four leaves of its plane,
//     leaf by leaf and column by column: for column j of leaf F0 F1 F2 F3,
//     v = F3 e_j and then F2, F1, F0 are applied to v (double-float
//     arithmetic), and v is added to column j of Q, kept in shared memory;
//     each warp handles one plane for 32 sites, so all its lanes take the
//     same path;
//  2. the entries of the two Hermitian 6x6 chiral blocks
//     1 + i kappa c_sw [[Gz, Gx - i Gy], [Gx + i Gy, -Gz]], with
//     Fhat = (Q - Q^dag) / 8, are packed and converted to FP64;
//  3. the stores in FP64, FP32 and FP16 (with the site norm).
constexpr int CL_SITES = 32;
constexpr int CL_THREADS = 6 * CL_SITES;

__global__ void __launch_bounds__(CL_THREADS) clover_build_kernel(Geom g, const float4 *Udf, double kappa, double csw,
                                                                   double2 *A64, float4 *A32, uint4 *A16, float *A16n,
                                                                   long long site0, long long site1)
{
    __shared__ float sQ[6][9][4][CL_SITES];  // Q per plane: [entry][re.h re.l im.h im.l][site]
    __shared__ double sP[72][CL_SITES];      // packed clover
    __shared__ double sN[CL_SITES];
    const long long V = g.V;
    const int t = threadIdx.x;
    {
        const int site = t % CL_SITES, plane = t / CL_SITES;
        const long long x = site0 + (long long)blockIdx.x * CL_SITES + site;
        if (x < site1) {
            // planes (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
            const int mu = (plane >= 3) + (plane >= 5);
            const int nu = plane < 3 ? plane + 1 : plane < 5 ? plane - 1 : 3;
            int c[4];
            site_coords(g, x, c);
#pragma unroll
            for (int k = 0; k < 9; k++)
#pragma unroll
                for (int q = 0; q < 4; q++) sQ[plane][k][q][site] = 0.f;
#pragma unroll 1
            for (int leaf = 0; leaf < 4; leaf++) {
                long long fx[4];
                int fd[4];
                bool fdag[4];
                leaf_factors(g, c, x, mu, nu, leaf, fx, fd, fdag);
                LinkFactor lf[4];
#pragma unroll
                for (int f = 0; f < 4; f++) lf[f] = link_factor((unsigned)V, fd[f], fx[f], fdag[f]);
#pragma unroll 1
                for (int j = 0; j < 3; j++) {
                    CDF v[3];  // column j of F3, then F2, F1, F0 applied to it
#pragma unroll
                    for (int a = 0; a < 3; a++) v[a] = lf_elem(Udf, lf[3], a, j);
                    // one copy of md_apply in the loop body keeps the hot code
                    // small enough for the instruction cache
#pragma unroll 1
                    for (int f = 2; f >= 0; f--) md_apply(Udf, lf[f], v);
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        float *e = &sQ[plane][a * 3 + j][0][site];
                        const DF qr = df_add(DF{e[0], e[CL_SITES]}, v[a].r);
                        const DF qi = df_add(DF{e[2 * CL_SITES], e[3 * CL_SITES]}, v[a].i);
                        e[0] = qr.h;
                        e[CL_SITES] = qr.l;
                        e[2 * CL_SITES] = qi.h;
                        e[3 * CL_SITES] = qi.l;
                    }
                }
            }
        }
    }
    __syncthreads();
    // packed blocks: h = 0 (spins 0,1) and 1 (spins 2,3), 6 diagonal reals and
    // 15 complex lower entries each
    const DF kc = df_from_double(kappa * csw);
    for (int w = t; w < 2 * 21 * CL_SITES; w += CL_THREADS) {
        const int site = w % CL_SITES, item = (w / CL_SITES) % 21, h = w / (21 * CL_SITES);
        int i, j;
        if (item < 6) {
            i = j = item;
        } else {  // lower entries in the packing order (1,0) (2,0) (2,1) (3,0) ...
            int r = item - 6;
            i = 1;
            while (r >= i) { r -= i; i++; }
            j = r;
        }
        const float sg = h == 0 ? -1.f : 1.f;
        const int s1 = i / 3, a = i % 3, s2 = j / 3, b = j % 3, k = a * 3 + b, kt = b * 3 + a;
        // Fhat_plane[a][b] = (Q_ab - conj(Q_ba)) / 8
        auto Fp = [&](int plane, int part) -> DF {
            const DF qa = DF{sQ[plane][k][2 * part][site], sQ[plane][k][2 * part + 1][site]};
            const DF qb = DF{sQ[plane][kt][2 * part][site], sQ[plane][kt][2 * part + 1][site]};
            return df_scale2(part == 0 ? df_sub(qa, qb) : df_add(qa, qb), 0.125f);
        };
        auto G = [&](int which, int part) -> DF {  // Gz = F_xy + sg F_zt, Gy = F_xz - sg F_yt, Gx = F_yz + sg F_xt
            if (which == 0) return df_add(Fp(0, part), df_scale2(Fp(5, part), sg));
            if (which == 1) return df_add(Fp(1, part), df_scale2(Fp(4, part), -sg));
            return df_add(Fp(3, part), df_scale2(Fp(2, part), sg));
        };
        DF br, bi;  // B_{s1 s2}[a][b]
        if (s1 == 0 && s2 == 0) { br = G(0, 0); bi = G(0, 1); }
        else if (s1 == 1 && s2 == 1) { br = df_neg(G(0, 0)); bi = df_neg(G(0, 1)); }
        else if (s1 == 0) { br = df_add(G(2, 0), G(1, 1)); bi = df_sub(G(2, 1), G(1, 0)); }   // Gx - i Gy
        else { br = df_sub(G(2, 0), G(1, 1)); bi = df_add(G(2, 1), G(1, 0)); }                // Gx + i Gy
        // M = delta + i kc B = delta + kc (-B.i + i B.r)
        DF mr = df_fma(kc, df_neg(bi), DF{0.f, 0.f});
        const DF mi = df_fma(kc, br, DF{0.f, 0.f});
        if (i == j) mr = df_add(mr, DF{1.f, 0.f});
        const int base = 36 * h;
        if (i == j) {
            sP[base + i][site] = df_to_double(mr);
        } else {
            sP[base + cl_off(i, j)][site] = df_to_double(mr);
            sP[base + cl_off(i, j) + 1][site] = df_to_double(mi);
        }
    }
    __syncthreads();
    if (t < CL_SITES) {
        double nrm = 0.0;
        for (int k = 0; k < 72; k++) nrm = fmax(nrm, fabs(sP[k][t]));
        sN[t] = nrm;
    }
    __syncthreads();
    for (int w = t; w < 36 * CL_SITES; w += CL_THREADS) {
        const int site = w % CL_SITES, k = w / CL_SITES;
        const long long x = site0 + (long long)blockIdx.x * CL_SITES + site;
        if (x >= site1) continue;
        A64[k * V + x] = make_double2(sP[2 * k][site], sP[2 * k + 1][site]);
        if (k < 18)
            A32[k * V + x] = make_float4((float)sP[4 * k][site], (float)sP[4 * k + 1][site], (float)sP[4 * k + 2][site],
                                         (float)sP[4 * k + 3][site]);
        if (k < 9) {
            const double nrm = sN[site];
            const float inv = nrm > 0 ? (float)(1.0 / nrm) : 0.f;
            unsigned wv[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                // word 4 k + q holds entry 4 k + q of both chiral blocks
                __half2 hh = __floats2half2_rn((float)sP[4 * k + q][site] * inv,
                                               (float)sP[36 + 4 * k + q][site] * inv);
                wv[q] = *reinterpret_cast<unsigned *>(&hh);
            }
            A16[k * V + x] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        if (k == 0) A16n[x] = (float)sN[site];
    }
}

cudaError_t launch_clover_build(const Geom &g, const void *Udf, double kappa, double csw, void *A64, void *A32,
                                void *A16, float *A16n, cudaStream_t st, long long site0, long long site1)
{
    if (site1 < 0) site1 = g.V;
    if (site1 <= site0) return cudaSuccess;
    const unsigned nb = (unsigned)((site1 - site0 + CL_SITES - 1) / CL_SITES);
    clover_build_kernel<<<nb, CL_THREADS, 0, st>>>(g, (const float4 *)Udf, kappa, csw, (double2 *)A64, (float4 *)A32,
                                            (uint4 *)A16, A16n, site0, site1);
    note_launch();
    return cudaGetLastError();
}

}  // namespace qdd
