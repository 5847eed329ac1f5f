// df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers with |lo| <= ulp(hi)/2, giving about 2^-47 relative
// precision on the FP32 pipes.
//
// Methods: Dekker, "A floating-point technique for extending the available
// precision" (Numer. Math. 18, 1971) for the representation and the fast
// two-sum; Knuth (TAOCP vol. 2) for the branch-free two-sum; Ogita, Rump and
// Oishi, "Accurate sum and dot product" (SIAM J. Sci. Comput. 26, 2005) for
// the FMA-based two-product.  Every step uses the _rn intrinsics so that the
// compiler neither contracts nor reorders the error-free transformations.
//
// Used where FP64 accuracy is needed but GB300's FP64 rate (about 1/74 of its
// FP32 rate) would dominate: the clover-term build and the SU(3) check of
// the gauge import.
#pragma once

namespace qdd {

struct DF {
    float h, l;
};

__device__ __forceinline__ DF df_from_double(double d)
{
    const float h = __double2float_rn(d);
    const float l = __double2float_rn(d - (double)h);
    return DF{h, l};
}

// Conversions between double and float in integer arithmetic: on this GPU
// the conversion instructions run on the FP64 pipe, at a small fraction of
// the integer rate, and they dominate kernels that convert many values.
// Biased double exponent of d.
__device__ __forceinline__ int dexp(double d) { return (__double2hiint(d) >> 20) & 0x7ff; }

// float(d) rounded to nearest even, exact for results in the normal float
// range (the 29 dropped mantissa bits decide the rounding; a carry out of the
// mantissa moves into the exponent, as IEEE 754 encodings allow); other
// inputs use the hardware conversion.
__device__ __forceinline__ float d2f_rn(double d)
{
    const int e = dexp(d);
    if (e < 897 || e > 1150) return __double2float_rn(d);
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    unsigned f = (hi & 0x80000000u) | ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu, half = 1u << 28;
    f += (rem > half || (rem == half && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
}

// double(f), exact; zeros, subnormals, infinities and NaNs use the hardware.
__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 255u) return (double)f;
    return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)),
                            (int)(b << 29));
}

// df_from_double with one FP64 operation (the exact subtraction d - hi).
__device__ __forceinline__ DF df_from_double_i(double d)
{
    const float h = d2f_rn(d);
    return DF{h, d2f_rn(d - f2d(h))};
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ DF fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = two_sum(a.h, b.h);
    const float t = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, t);
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }

__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

// c + a b
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);           // p + e = a.h b.h exactly (Ogita-Rump-Oishi)
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    DF s = two_sum(p, c.h);
    const float t = __fadd_rn(s.l, __fadd_rn(e, c.l));
    return fast_two_sum(s.h, t);
}

// Scaling by a power of two is exact.
__device__ __forceinline__ DF df_scale2(DF a, float pow2) { return DF{a.h * pow2, a.l * pow2}; }

// Accumulator for a sum of double-float products, after the Dot2 algorithm
// of Ogita, Rump and Oishi (same paper): the products' high parts are summed
// with two_sum, and every rounding error, together with the products' cross
// terms, is gathered in one FP32 correction that is folded in at the end.
// 12 instructions per product instead of 14 for a chain of df_fma.
struct DFAcc {
    float s, c;
};

__device__ __forceinline__ void dfacc_init(DFAcc &a, DF x, DF y)  // a = x y
{
    a.s = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -a.s);
    e = __fmaf_rn(x.h, y.l, e);
    a.c = __fmaf_rn(x.l, y.h, e);
}

__device__ __forceinline__ void dfacc_add(DFAcc &a, DF x, DF y)  // a += x y
{
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    const DF t = two_sum(a.s, p);
    a.s = t.h;
    a.c = __fadd_rn(a.c, __fadd_rn(t.l, e));
}

__device__ __forceinline__ DF dfacc_result(const DFAcc &a) { return two_sum(a.s, a.c); }

struct CDF {
    DF r, i;
};

// c + a b (complex)
__device__ __forceinline__ CDF cdf_fma(CDF a, CDF b, CDF c)
{
    c.r = df_fma(a.r, b.r, c.r);
    c.r = df_fma(df_neg(a.i), b.i, c.r);
    c.i = df_fma(a.r, b.i, c.i);
    c.i = df_fma(a.i, b.r, c.i);
    return c;
}

// c + conj(a) b
__device__ __forceinline__ CDF cdf_fma_ca(CDF a, CDF b, CDF c)
{
    c.r = df_fma(a.r, b.r, c.r);
    c.r = df_fma(a.i, b.i, c.r);
    c.i = df_fma(a.r, b.i, c.i);
    c.i = df_fma(df_neg(a.i), b.r, c.i);
    return c;
}

// c + a conj(b)
__device__ __forceinline__ CDF cdf_fma_cb(CDF a, CDF b, CDF c)
{
    c.r = df_fma(a.r, b.r, c.r);
    c.r = df_fma(a.i, b.i, c.r);
    c.i = df_fma(df_neg(a.r), b.i, c.i);
    c.i = df_fma(a.i, b.r, c.i);
    return c;
}

}  // namespace qdd
