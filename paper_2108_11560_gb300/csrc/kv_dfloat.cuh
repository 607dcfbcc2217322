// Float-float ("double-float") arithmetic on the FP32 pipe: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits.  Error-free transformations after Dekker (1971) and Knuth (TAOCP
// vol. 2): TwoSum, FastTwoSum and TwoProd (the latter with one fused multiply-add).
//
// GB300 runs FP64 at about 1/70 of the FP32 rate (a measured FP64 exp costs ~140 FP32 expf), so
// the extended-precision work of the learned-bracket path (the offset g(t_r) and the per-pair
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

// x + y with the low parts added in FP32 (Dekker's addition): the high parts are summed
// exactly, so cancellation between them costs nothing; relative error about 2^-44 unless the
// low parts themselves cancel.
__device__ __forceinline__ df df_add_fast(df x, df y)
{
    df s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_sub_fast(df x, df y) { return df_add_fast(x, df_neg(y)); }

// x + y and x - y as df_add_fast, for |x.hi| >= |y.hi| (FastTwoSum on the high parts).
__device__ __forceinline__ df df_add_ordered(df x, df y)
{
    df s = fast_two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_sub_ordered(df x, df y) { return df_add_ordered(x, df_neg(y)); }

// ln 2 as a float-float.
__device__ __forceinline__ df df_ln2() { return df{0.6931472f, -1.9046542e-09f}; }

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

}  // namespace kvd
