// Float-float ("double-float") arithmetic on the FP32 pipe: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits.  Error-free transformations after Dekker (1971) and Knuth (TAOCP
// vol. 2): TwoSum, FastTwoSum and TwoProd (the latter with one fused multiply-add).
//
// GB300 runs FP64 at about 1/70 of the FP32 rate (a measured FP64 exp costs ~140 FP32 expf), so
// the extended-precision work of the learned-bracket path (the offset g(t_p) and the per-pair
// constants whose inputs cancel) is done here instead of in FP64.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace kvd {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return df{a, 0.0f}; }

// s + e = a + b exactly (any a, b).
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// s + e = a + b exactly, valid when |a| >= |b| or a == 0.
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

// p + e = a * b exactly.
__device__ __forceinline__ df two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = fmaf(a, b, -p);
    return df{p, e};
}

__device__ __forceinline__ df df_add(df x, df y)
{
    df s = two_sum(x.hi, y.hi);
    df t = two_sum(x.lo, y.lo);
    float e = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, e);
    e = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y)
{
    df p = two_prod(x.hi, y.hi);
    float e = fmaf(x.hi, y.lo, p.lo);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_mul_f(df x, float f)
{
    df p = two_prod(x.hi, f);
    float e = fmaf(x.lo, f, p.lo);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_scale2(df x, int k) { return df{ldexpf(x.hi, k), ldexpf(x.lo, k)}; }

// 1 / y by one Newton step r' = r + r (1 - y r) from the FP32 reciprocal (doubles the bits).
__device__ __forceinline__ df df_rcp(df y)
{
    float r = __frcp_rn(y.hi);
    df e = df_sub(df_make(1.0f), df_mul_f(y, r));  // 1 - y r
    return df_add(df_make(r), df_mul_f(e, r));
}

// e^t for FP32 t as a float-float, relative error about 1e-13 for |t| < 80.
// Cody & Waite (1980) reduction t = k ln2 + r with ln2 split in three floats (the first with few
// significant bits, so k * LN2_A is exact), |r| <= ln2/2; e^r by its Taylor series, the terms up
// to r^5 in float-float and r^6..r^12 in FP32 (they are below 2.3e-6 of the sum); then 2^k.
__device__ __forceinline__ df df_exp(float t)
{
    constexpr float LN2_A = 0.693145751953125f;  // 16 significant bits: k * LN2_A is exact
    constexpr float LN2_B = 1.4286068e-06f;       // ln2 - A rounded
    constexpr float LN2_C = 5.497923e-14f;        // ln2 - A - B rounded
    float k = rintf(t * 1.4426950408889634f);
    float r0 = fmaf(-k, LN2_A, t);                 // exact (Sterbenz)
    df r = df_sub(df_make(r0), two_prod(k, LN2_B));
    r = df_sub(r, df_make(k * LN2_C));
    // tail: sum_{j>=6} r^j / j! = r^6 q(r), in FP32
    float rh = r.hi;
    float q = 1.0f / 479001600.0f;                 // 1/12!
    q = fmaf(q, rh, 1.0f / 39916800.0f);
    q = fmaf(q, rh, 1.0f / 3628800.0f);
    q = fmaf(q, rh, 1.0f / 362880.0f);
    q = fmaf(q, rh, 1.0f / 40320.0f);
    q = fmaf(q, rh, 1.0f / 5040.0f);
    q = fmaf(q, rh, 1.0f / 720.0f);
    float r2 = rh * rh;
    float tail = q * (r2 * r2 * r2);
    // head: 1 + r + r^2/2 + r^3/6 + r^4/24 + r^5/120 by Horner in float-float
    const df c5 = df{0.008333334f, -4.346172e-10f};  // 1/120
    const df c4 = df{0.041666668f, -1.2417635e-09f}; // 1/24
    const df c3 = df{0.16666667f, -4.967054e-09f};   // 1/6
    df p = c5;
    p = df_add(df_mul(p, r), c4);
    p = df_add(df_mul(p, r), c3);
    p = df_add(df_mul(p, r), df_make(0.5f));
    p = df_add(df_mul(p, r), df_make(1.0f));
    p = df_add(df_mul(p, r), df_make(1.0f));
    p = df_add(p, df_make(tail));
    return df_scale2(p, (int)k);
}

// ln 2 as a float-float.
__device__ __forceinline__ df df_ln2() { return df{0.6931472f, -1.9046542e-09f}; }

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

}  // namespace kvd
