// Float-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2 (48-bit significand, FP32 exponent range).  Sums use Knuth's error-free two-sum,
// products the FMA two-product (Dekker 1971; the double-double scheme of Hida, Li and Bailey, 2001),
// so every operation is a handful of FP32 instructions on pipes that run ~60x the FP64 rate of this
// part.  In namespace fef::ffa so that its fma overload does not hide the math library's in fef.
#pragma once

#include <cuda_runtime.h>

namespace fef {
namespace ffa {

struct df64 {
    float hi, lo;
    df64() = default;
    __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit df64(int i) : hi((float)i), lo(0.0f) {}
};

__device__ __forceinline__ df64 quick_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df64(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    const df64 t = two_sum(a.hi, b.hi);
    return quick_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}

// a b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df64 t = two_sum(p, c.hi);
    return quick_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(e, c.lo)));
}

// 1/sqrt(x), x > 0: float seed, one float Newton step, one df64 Newton step (relative error ~1e-14).
__device__ __forceinline__ df64 rsqrt_df(df64 x)
{
    float r = rsqrtf(x.hi);
    r = r * (1.5f - 0.5f * x.hi * r * r);
    const df64 y(r, 0.0f);
    const df64 e = df64(1.0f, 0.0f) - x * (y * y);  // ~1e-7
    return quick_two_sum(r, 0.5f * r * e.hi);
}

// a b for a df64 a and a float b
__device__ __forceinline__ df64 mul_f(df64 a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return quick_two_sum(p, e);
}

// FP64 <-> float-float
__device__ __forceinline__ df64 from_double(double v)
{
    const float h = (float)v;
    return df64(h, (float)(v - (double)h));
}
__device__ __forceinline__ double to_double(df64 v) { return (double)v.hi + (double)v.lo; }

// Sum of df64 products kept unnormalised (s + c): each product x y adds its rounded leading part to s
// by Knuth's two-sum and its error terms (the FMA residual of x.hi y.hi and the cross products) to c,
// with no renormalisation per term (the compensated dot product of Ogita, Rump and Oishi, 2005);
// 12 FP32 operations per term instead of 15 for a normalised df64 fma.
struct dfacc {
    float s, c;
};

__device__ __forceinline__ void acc_prod(dfacc& a, df64 x, df64 y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    const float s = __fadd_rn(a.s, p);
    const float bp = __fsub_rn(s, a.s);
    const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(t, e));
}

}  // namespace ffa
}  // namespace fef
