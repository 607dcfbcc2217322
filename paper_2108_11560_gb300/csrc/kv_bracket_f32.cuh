// FP32 range finding for one (v, x) pair: Algorithms 1-3 (Sec. 2.1-2.3) in single precision, the
// bracket of the paper's 32-bit variant (Sec. 4.2).
//
// The searches are those of kv_bracket.cuh (same readings: FindZero keeps the end where F < 0,
// takes the bisection point and the clipped Newton point each iteration and returns the negative
// end after exactly max_iter iterations; FindRange doubles from m = 0).  What changes is how the
// functions are evaluated so that FP32 suffices:
//  * the peak search works on g'(t) = v tanh(vt) - x sinh t and g''(t) directly (their zero and
//    sign need only FP32 relative accuracy of the two terms);
//  * the range searches work on h(t) = g(t) - g(t_r) - log eps through the cancellation-free
//    difference of kv_bins.cuh about a reference point t_r next to the peak (the caller supplies
//    the per-pair constants at t_r), in its coarse form (absolute error about 2^-22 of
//    x e^{+-t_r}/2), instead of losing |g| 2^-24 to the subtraction of two large numbers.
//    g(t_r) <= g(t_p) by at most a fraction of a nat (t_r is within ln2/256 of the FP32 peak),
//    which widens the range by that much.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "kv_bins.cuh"

namespace kvd {

constexpr int KV_RANGE_CAP_F32 = 11;

// sinh t and cosh t for t >= 0 in FP32: a short series below 1/2 (where e^t - e^-t cancels),
// ex2 and its reciprocal above.
__device__ __forceinline__ void sinh_cosh_f32(float t, float& sh, float& ch)
{
    const float et = ex2_approx(t * LOG2E_F), eti = rcp_approx(et);
    const float z = t * t;
    const float ss = t * fmaf(z, fmaf(z, fmaf(z, 1.0f / 5040.0f, 1.0f / 120.0f), 1.0f / 6.0f), 1.0f);
    sh = t < 0.5f ? ss : 0.5f * (et - eti);
    ch = 0.5f * (et + eti);
}

// F = g'(t), F' = g''(t) (the peak search).
__device__ __forceinline__ void eval_g1_g2_f32(float v, float x, float t, float& F, float& dF)
{
    const float vt = v * t;
    const float e2 = ex2_approx(-2.0f * LOG2E_F * vt);
    const float r = rcp_approx(1.0f + e2);
    const float th = vt < TANH_SERIES_MAX ? tanh_small(vt) : (1.0f - e2) * r;
    float sh, ch;
    sinh_cosh_f32(t, sh, ch);
    F = v * th - x * sh;
    dF = v * v * (4.0f * e2 * r * r) - x * ch;
}

// F = h(t) = g(t_r + s) - g(t_r) - log eps with s = t - t_r, F' = g'(t) (the range searches),
// from the coarse form of the same cancellation-free difference that the learned path's range
// check uses (kv_bins.cuh delta_g_coarse: phi(+-s) = e^{+-s} - 1 -+ s from the approximate
// exponential, no series).  Its error, about 2^-22 of x e^{+-t_r}/2 in absolute terms, moves the
// range's ends by a vanishing fraction of a nat of the eps level; the searches need only the sign
// of h and a usable slope.
__device__ __forceinline__ void eval_h_f32(const BinsF& b, float le, float t, float& F, float& dF)
{
    float e2, es, ems;
    F = delta_g_coarse(b, t - b.tp, e2, es, ems) - le;
    dF = delta_g_slope_f32(b, e2, es, ems);
}

template <int KIND>
__device__ __forceinline__ void eval_F_f32(float v, float x, const BinsF& b, float le, float t, float& F,
                                           float& dF)
{
    if (KIND == 0) eval_g1_g2_f32(v, x, t, F, dF);
    else eval_h_f32(b, le, t, F, dF);
}

// The same functions at two points at once (the bisection and Newton points of one FindZero
// iteration), in paired FP32 instructions.
__device__ __forceinline__ void eval_g1_g2_f32x2(float v, float x, float2 t, float2& F, float2& dF)
{
    const float2 vt = mul2(f2(v), t);
    const float2 ea = mul2(vt, f2(-2.0f * LOG2E_F));
    const float2 e2 = make_float2(ex2_approx(ea.x), ex2_approx(ea.y));
    const float2 ope = add2(f2(1.0f), e2);
    const float2 r = make_float2(rcp_approx(ope.x), rcp_approx(ope.y));
    const float2 thl = mul2(fma2(e2, f2(-1.0f), f2(1.0f)), r);
    const float2 thz = mul2(vt, vt);
    float2 thp;
    KV_TANH_POLY(fma2, f2, thz, thp)
    const float2 ths = fma2(mul2(vt, thz), thp, vt);
    const float2 th = make_float2(vt.x < TANH_SERIES_MAX ? ths.x : thl.x, vt.y < TANH_SERIES_MAX ? ths.y : thl.y);
    const float2 el = mul2(t, f2(LOG2E_F));
    const float2 et = make_float2(ex2_approx(el.x), ex2_approx(el.y));
    const float2 eti = make_float2(rcp_approx(et.x), rcp_approx(et.y));
    const float2 z = mul2(t, t);
    const float2 ss = mul2(t, fma2(z, fma2(z, fma2(z, f2(1.0f / 5040.0f), f2(1.0f / 120.0f)), f2(1.0f / 6.0f)), f2(1.0f)));
    const float2 shl = mul2(fma2(eti, f2(-1.0f), et), f2(0.5f));
    const float2 sh = make_float2(t.x < 0.5f ? ss.x : shl.x, t.y < 0.5f ? ss.y : shl.y);
    const float2 ch = mul2(add2(et, eti), f2(0.5f));
    F = fma2(f2(v), th, mul2(f2(-x), sh));
    dF = fma2(f2(v * v), mul2(mul2(f2(4.0f), e2), mul2(r, r)), mul2(f2(-x), ch));
}

template <int KIND>
__device__ __forceinline__ void eval_F_f32x2(float v, float x, const BinsF& b, float le, float2 t, float2& F,
                                             float2& dF)
{
    if (KIND == 0) {
        eval_g1_g2_f32x2(v, x, t, F, dF);
    } else {
        float2 e2, es, ems;
        F = add2(delta_g_coarse2(b, add2(t, f2(-b.tp)), e2, es, ems), f2(-le));
        dF = delta_g_slope2(b, e2, es, ems);
    }
}

// Algorithm 1 in FP32; returns false when the doubling cap was hit before the sign changed.
template <int KIND>
__device__ __forceinline__ bool find_range_f32(float v, float x, const BinsF& b, float le, float t0,
                                               float& t_pos, float& t_neg, float& F_neg, float& dF_neg)
{
    int m = 0;
    float F, dF;
    eval_F_f32<KIND>(v, x, b, le, t0 + 2.0f, F, dF);
    while (m < KV_RANGE_CAP_F32 && F >= 0.0f) {
        ++m;
        eval_F_f32<KIND>(v, x, b, le, t0 + ldexpf(1.0f, m + 1), F, dF);
    }
    float lo = t0 + ldexpf(1.0f, m);
    if (m == 0) {
        float Flo, dFlo;
        eval_F_f32<KIND>(v, x, b, le, lo, Flo, dFlo);
        if (!(Flo >= 0.0f)) lo = t0;
    }
    t_pos = lo;
    t_neg = t0 + ldexpf(1.0f, m + 1);
    F_neg = F;
    dF_neg = dF;
    return F < 0.0f;
}

// Algorithm 2 in FP32 with a fixed trip count.  Each iteration evaluates F at both the bisection
// point and the Newton point, together in paired instructions, and selects the update with
// predicates (the Newton point's value is used only where the bisection point is on the positive
// side, as in the algorithm): lanes of a warp that would take different sides of the test then
// run the same instructions instead of running the two sides one after the other.
template <int KIND>
__device__ __forceinline__ float find_zero_f32(float v, float x, const BinsF& b, float le, float t_neg,
                                               float t_pos, float Fa, float dFa, int max_iter)
{
    float a = t_neg, bb = t_pos;
    for (int i = 0; i < max_iter; ++i) {
        const float shrink = a + (bb - a) * 0.5f;
        float newton = a - __fdividef(Fa, dFa);
        newton = isfinite(newton) ? newton : shrink;
        newton = fminf(fmaxf(newton, fminf(t_neg, shrink)), fmaxf(t_neg, shrink));
        float2 F2, dF2;
        eval_F_f32x2<KIND>(v, x, b, le, make_float2(shrink, newton), F2, dF2);
        const float Fs = F2.x, dFs = dF2.x, Fn = F2.y, dFn = dF2.y;
        const bool s_neg = Fs < 0.0f;           // the bisection point becomes the negative end
        const bool n_neg = !s_neg && Fn < 0.0f;  // else the Newton point does, if negative
        a = s_neg ? shrink : (n_neg ? newton : a);
        Fa = s_neg ? Fs : (n_neg ? Fn : Fa);
        dFa = s_neg ? dFs : (n_neg ? dFn : dFa);
        bb = s_neg ? bb : (n_neg ? shrink : newton);
    }
    return a;
}

// Algorithm 2 in FP32 for both ends of the range at once: once the peak is known the t0 search on
// [0, t_p] and the t1 search after FindRange are independent, so they run as the two components
// of float2 iterates (x: t0, y: t1), each component taking exactly find_zero_f32's steps; the four
// points of an iteration are evaluated as two pairs.  A pair whose t0 search is not needed runs it
// on its placeholder end points (the result is not used), so that the warp runs one loop.
__device__ __forceinline__ float2 find_zero2_f32(const BinsF& b, float le, float2 t_neg, float2 t_pos,
                                                 float2 Fa, float2 dFa, int max_iter)
{
    float2 a = t_neg, bb = t_pos;
    for (int i = 0; i < max_iter; ++i) {
        const float2 shrink = fma2(fma2(a, f2(-1.0f), bb), f2(0.5f), a);
        float2 newton = fma2(make_float2(-Fa.x, -Fa.y), make_float2(rcp_approx(dFa.x), rcp_approx(dFa.y)), a);
        newton.x = isfinite(newton.x) ? newton.x : shrink.x;
        newton.y = isfinite(newton.y) ? newton.y : shrink.y;
        newton.x = fminf(fmaxf(newton.x, fminf(t_neg.x, shrink.x)), fmaxf(t_neg.x, shrink.x));
        newton.y = fminf(fmaxf(newton.y, fminf(t_neg.y, shrink.y)), fmaxf(t_neg.y, shrink.y));
        float2 F0, dF0, F1, dF1;  // (shrink, newton) of the t0 search, then of the t1 search
        eval_F_f32x2<1>(0.0f, 0.0f, b, le, make_float2(shrink.x, newton.x), F0, dF0);
        eval_F_f32x2<1>(0.0f, 0.0f, b, le, make_float2(shrink.y, newton.y), F1, dF1);
        const bool s0 = F0.x < 0.0f, n0 = !s0 && F0.y < 0.0f;
        const bool s1 = F1.x < 0.0f, n1 = !s1 && F1.y < 0.0f;
        a = make_float2(s0 ? shrink.x : (n0 ? newton.x : a.x), s1 ? shrink.y : (n1 ? newton.y : a.y));
        Fa = make_float2(s0 ? F0.x : (n0 ? F0.y : Fa.x), s1 ? F1.x : (n1 ? F1.y : Fa.y));
        dFa = make_float2(s0 ? dF0.x : (n0 ? dF0.y : dFa.x), s1 ? dF1.x : (n1 ? dF1.y : dFa.y));
        bb = make_float2(s0 ? bb.x : (n0 ? shrink.x : newton.x), s1 ? bb.y : (n1 ? shrink.y : newton.y));
    }
    return a;
}

// Algorithm 3's peak in FP32 (0 when v^2 <= x).
__device__ __forceinline__ float peak_alg12_f32(float v, float x, int max_iter, bool& capped)
{
    if (!(v * v - x > 0.0f)) return 0.0f;
    BinsF unused;
    float ts, te, F, dF;
    capped |= !find_range_f32<0>(v, x, unused, 0.0f, 0.0f, ts, te, F, dF);
    return find_zero_f32<0>(v, x, unused, 0.0f, te, ts, F, dF, max_iter);
}

// Algorithm 3's range [t0, t1] in FP32, given the peak tp and the per-pair constants b at the
// reference point b.tp (s0, h and n of b are not used).  Returns false if the result is not a
// finite range with 0 <= t0 <= t1.
__device__ __forceinline__ bool range_alg12_f32(const BinsF& b, float tp, float le, int max_iter,
                                                float& t0, float& t1, bool& capped)
{
    float h0, dh0;
    eval_h_f32(b, le, 0.0f, h0, dh0);
    const bool left = tp > 0.0f && h0 <= 0.0f;  // the range does not reach t = 0
    float ts, te, F, dF;
    capped |= !find_range_f32<1>(0.0f, 0.0f, b, le, tp, ts, te, F, dF);
    // t0 on [0, t_p] (negative end 0) and t1 on FindRange's bracket, together
    const float2 r = find_zero2_f32(b, le, make_float2(0.0f, te), make_float2(left ? tp : 1.0f, ts),
                                    make_float2(left ? h0 : -1.0f, F), make_float2(left ? dh0 : 1.0f, dF), max_iter);
    t0 = left ? r.x : 0.0f;
    t1 = r.y;
    return isfinite(t0) && isfinite(t1) && t0 >= 0.0f && t1 > t0;
}

}  // namespace kvd
