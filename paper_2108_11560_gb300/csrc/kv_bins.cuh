// The fixed-bin trapezoid sums of Sec. 2.4 (Eq. int) and Sec. 4.1, for one pair, split over
// L lanes of a warp (lane l takes bins l, l + L, ...).
//
// Every bin m in 0..n has t_m = t0 + m h and weight c_m exp(g(t_m) - g(t_p)), c_0 = c_n = 1/2.
// Three sums share the weights:  S0 = sum w,  S1 = sum w t tanh(vt),  S2 = sum w cosh t.
// Then log K = g(t_p) + log h + log S0,  d/dv log K = S1 / S0,  d/dx log K = -S2 / S0.
//
// The difference g(t_m) - g(t_p) is never formed by subtracting two large values.  With
// s = t - t_p and u = v t_p (t, t_p >= 0):
//   log cosh(vt) - log cosh(u) = v s + log1p(e^{-2vt}) - log1p(e^{-2u})
//   x (cosh t - cosh t_p)      = x sinh(t_p) s + (x e^{t_p}/2) phi(s) + (x e^{-t_p}/2) phi(-s)
//                                with phi(s) = e^s - 1 - s >= 0
//                              ( = 2 x sinh((t + t_p)/2) sinh(s/2), used by the FP64 second-
//                                derivative sums)
// so that every term is small where the weight is large and no two large terms cancel:
//   g(t) - g(t_p) = (v - x sinh t_p) s + [log1p(e^{-2vt}) - log1p(e^{-2u})]
//                   - (x e^{t_p}/2) phi(s) - (x e^{-t_p}/2) phi(-s).
// The per-pair constants (v - x sinh t_p, x e^{+-t_p}/2, log1p(e^{-2u}), g(t_p)) carry extra
// precision: FP64 with the plain bracket, float-float with the learned one.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <math.h>

namespace kvd {

constexpr float LOG2E_F = 1.4426950408889634f;
constexpr float LN2_F = 0.6931471805599453f;

__device__ __forceinline__ float ex2_approx(float a)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float lg2_approx(float a)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// Compensated (Kahan) accumulation.
template <typename T>
struct KahanSum {
    T s, c;
    __device__ __forceinline__ void init() { s = T(0); c = T(0); }
    __device__ __forceinline__ void add(T w)
    {
        T y = w - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ T value() const { return s - c; }
};

template <typename T, int L>
__device__ __forceinline__ T lane_sum(T a)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o, L);
    return a;
}

// ------------------------------------------------------------------ FP64 bins

struct BinsD {
    double v, x, t0, h, tp, s0, Lu;  // s0 = t0 - t_p, Lu = log1p(e^{-2 v t_p})
    double e2u;                      // e^{-2 v t_p}
    double ep, em;                   // e^{t_p}, e^{-t_p}
    double c1;                       // v - x sinh t_p
    double xch, xsh;                 // x cosh t_p, x sinh t_p
    double shp;                      // sinh t_p
    int n;
};

// E(z) = (cosh s - 1)/z and O(z) = (sinh s / s - 1)/z, z = s^2 <= 1, as degree-6 minimax
// polynomials (minimax_coeffs.py: absolute errors 5.9e-18 and 3.5e-19, below double rounding);
// phi(+-s) = e^{+-s} - 1 -+ s = z (E +- s O).
__device__ __forceinline__ void phi_parts_f64(double z, double& E, double& O)
{
    E = 1.1639213882575488e-11;
    E = fma(E, z, 2.087443498312207e-9);
    E = fma(E, z, 2.7557335075601938e-7);
    E = fma(E, z, 2.4801587246062242e-5);
    E = fma(E, z, 1.3888888888981485e-3);
    E = fma(E, z, 4.1666666666666088e-2);
    E = fma(E, z, 0.5);
    O = 7.7461889806431037e-13;
    O = fma(O, z, 1.6057679312178728e-10);
    O = fma(O, z, 2.5052117699413503e-8);
    O = fma(O, z, 2.755731919136364e-6);
    O = fma(O, z, 1.9841269841324241e-4);
    O = fma(O, z, 8.3333333333332993e-3);
    O = fma(O, z, 0.16666666666666667);
}

// e^{+-s} and e^{-2vt} advance by one multiplication per bin and are recomputed exactly every
// this many steps, so their relative error stays below this many ulps.
constexpr int kRefreshF64 = 32;

// FP64 bins, one transcendental per bin (the weight's exp).  With s = t - t_p and u = v t_p,
//   g(t) - g(t_p) = c1 s + [log1p(e^{-2vt}) - log1p(e^{-2u})] + N(s),
//   c1 = v - x sinh t_p,  N(s) = -(x e^{t_p}/2) phi(s) - (x e^{-t_p}/2) phi(-s),  phi(s) = e^s - 1 - s,
// and the weight is taken as e^{g(t) - g(t_p)} = (1 + e^{-2vt}) / (1 + e^{-2u}) exp(c1 s + N(s)),
// so no log1p is evaluated; the tanh integrand is w tanh(vt) = (1 - e^{-2vt}) / (1 + e^{-2u})
// exp(...), with 1 - e^{-2vt} = -expm1(-2vt) below vt = 1/2 (no cancellation) and no division.
// phi(+-s) = z (E(z) +- s O(z)), z = s^2, for |s| <= 1 with E = (cosh s - 1)/z and
// O = (sinh s / s - 1)/z as degree-6 minimax polynomials on z in [0, 1] (minimax_coeffs.py:
// absolute errors 5.9e-18 and 3.5e-19, below double rounding), so
// N = -z (x cosh t_p E + x sinh t_p s O); beyond, from e^{+-s}, where e^s - 1 - s loses at most a
// factor e/phi(1) < 4 of e^s's accuracy.  The cosh t integrand is (e^{t_p} e^s + e^{-t_p} e^{-s})/2,
// a sum of positive terms.  The three sums are plain within each block of kRefreshF64 steps
// (relative error below 31 ulps: all terms are positive) and compensated (Kahan) across blocks,
// so the summation error does not grow with the bin count.
template <int L, bool DERIV>
__device__ __forceinline__ void sums_f64(const BinsD& b, int lane, double& S0, double& S1, double& S2)
{
    KahanSum<double> k0, k1, k2;
    k0.init();
    k1.init();
    k2.init();
    double p0 = 0.0, p1 = 0.0, p2 = 0.0;  // this block's plain sums
    const double kc = 1.0 / (1.0 + b.e2u);  // e^{-log1p(e^{-2u})}
    const double ap = 0.5 * b.x * b.ep, am = 0.5 * b.x * b.em;
    const double step = L * b.h;
    const double qs = exp(step), qsi = exp(-step), q2 = exp(-2.0 * b.v * step);
    double es = 1.0, esi = 1.0, e2 = 1.0;
    int since = kRefreshF64;
    for (int m = lane; m <= b.n; m += L) {
        const double s = fma((double)m, b.h, b.s0);
        const double t = b.tp + s;
        if (since == kRefreshF64) {
            es = exp(s);
            esi = 1.0 / es;
            e2 = exp(-2.0 * b.v * t);
            since = 0;
            k0.add(p0);
            k1.add(p1);
            k2.add(p2);
            p0 = p1 = p2 = 0.0;
        }
        const double z = s * s;
        double E, O;
        phi_parts_f64(z, E, O);
        const double n_small = -z * fma(b.xch, E, b.xsh * (s * O));
        const double n_large = fma(b.xsh, s, b.xch) - fma(ap, es, am * esi);
        const double N = fabs(s) <= 1.0 ? n_small : n_large;
        const double c = (m == 0 || m == b.n) ? 0.5 : 1.0;
        const double wp = c * kc * exp(fma(b.c1, s, N));
        // rounded products and sums (never contracted into an FMA), so that log K comes out the
        // same bits with and without the derivative sums
        const double w = __dmul_rn(wp, 1.0 + e2);
        p0 = __dadd_rn(p0, w);
        if (DERIV) {
            const double vt = b.v * t;
            double q = 1.0 - e2;  // (1 + e^{-2vt}) tanh(vt)
            if (vt < 0.5) q = -expm1(-2.0 * vt);
            p1 = fma(wp, t * q, p1);
            const double ch = 0.5 * fma(b.ep, es, b.em * esi);  // cosh t
            p2 += w > 0.0 ? w * ch : 0.0;
        }
        es *= qs;
        esi *= qsi;
        e2 *= q2;
        ++since;
    }
    k0.add(p0);
    k1.add(p1);
    k2.add(p2);
    S0 = lane_sum<double, L>(k0.value());
    S1 = DERIV ? lane_sum<double, L>(k1.value()) : 0.0;
    S2 = DERIV ? lane_sum<double, L>(k2.value()) : 0.0;
}

// ------------------------------------------------------------------ FP32 bins

struct BinsF {
    float s0, h;    // s_m = s0 + m h
    float v, u, tp; // |v|, v t_p, t_p
    float c1;       // v - x sinh t_p
    float ap, am;   // x e^{t_p} / 2, x e^{-t_p} / 2
    float lu;       // log1p(e^{-2u})
    float ep, em;   // e^{t_p}, e^{-t_p}
    float e2u, shp; // e^{-2u}, sinh t_p (second derivatives only)
    float xch, xsh; // x cosh t_p, x sinh t_p
    int n;
};

// Blackwell executes FP32 add, multiply and fused multiply-add on pairs of values (f32x2) at one
// issue slot per pair; the bins were issue-bound, so two bins of a lane go through the same
// arithmetic as one float2 (each component rounds exactly like the scalar instruction).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// phi(s) = e^s - 1 - s and phi(-s), and e^{+-s}.
// |s| <= 1: phi(+-s) = z (E(z) +- s O(z)) with z = s^2 and the even/odd parts
//   E(z) = (cosh s - 1) / z = sum_{k>=1} z^{k-1}/(2k)!,  O(z) = (sinh s / s - 1) / z = sum_{k>=1} z^{k-1}/(2k+1)!,
// each replaced by its degree-3 minimax polynomial on z in [0, 1] (Remez exchange; the script
// minimax_coeffs.py beside this file prints the coefficients): absolute errors 2.2e-9 (E, about
// 0.5) and 2.0e-10 (O, about 1/6), below FP32 rounding, where the Taylor polynomials of the same
// degree leave 2.8e-7 and 2.5e-8.
// |s| > 1: from e^s = 2^{s log2 e} (ex2.approx: relative error about 2^-22 plus the rounding of
// s log2 e, |s| 2^-24 relative), where the cancellation in e^s - 1 - s costs at most a few ulps of
// e (phi(1) = 0.718, phi(-1) = 0.368: relative error below 1e-6 at |s| = 1, falling beyond).  The
// weight of such a bin is exp(-(x e^{t_p}/2) phi(s) - ...), so the absolute error this leaves in
// its exponent stays below 1e-6 wherever the bin's weight is not negligible.
// Both forms are computed and the valid one is selected: lanes of a warp whose bins straddle
// |s| = 1 would otherwise run both sides one after the other.  (The polynomial at |s| > 1 is
// discarded; it stays finite far beyond any range the bins cover, and an overflow there would
// not reach the selected value.)  e^{+-s} themselves (for cosh t in the d/dx integrand, which
// needs only FP32 relative accuracy) always come from ex2 and its reciprocal.
constexpr float PHI_SERIES_MAX = 1.0f;

#define KV_PHI_SERIES(MUL, FMA, C, z, E, O)                        \
    E = FMA(C(2.5358777544656039e-5f), z, C(1.3885392932591772e-3f)); \
    E = FMA(E, z, C(4.1666736744439945e-2f));                        \
    E = FMA(E, z, C(0.5f));                                          \
    O = FMA(C(2.8063006223552967e-6f), z, C(1.9838098914288133e-4f)); \
    O = FMA(O, z, C(8.3333396873695536e-3f));                        \
    O = FMA(O, z, C(0.16666666646778531f));

__device__ __forceinline__ float f1(float a) { return a; }

__device__ __forceinline__ void phi_pair(float s, float& php, float& phm, float& es, float& ems)
{
    const float z = s * s;
    float E, O;
    KV_PHI_SERIES(__fmul_rn, fmaf, f1, z, E, O)
    const float so = s * O;
    const float pp = z * (E + so), pm = z * (E - so);
    es = ex2_approx(s * LOG2E_F);
    ems = rcp_approx(es);
    const bool small = fabsf(s) <= PHI_SERIES_MAX;
    php = small ? pp : (es - 1.0f) - s;
    phm = small ? pm : (ems - 1.0f) + s;
}

// tanh(y) for |y| < 0.35 as y + y^3 P(y^2), P the degree-3 minimax polynomial of
// (tanh(y)/y - 1)/y^2 on y^2 in [0, 0.35^2] (absolute error 1.4e-8 in P, so tanh's relative
// error is below 2e-9 before FP32 rounding; coefficients from minimax_coeffs.py);
// (1 - e^{-2y}) / (1 + e^{-2y}) loses relative precision to the cancellation in 1 - e^{-2y}
// (about 2^-22 / (2y) relative: below 4e-7 from y = 0.35 on).
#define KV_TANH_POLY(FMA, C, z, p)                      \
    p = FMA(C(1.9843806701481164e-2f), z, C(-5.3817014230769577e-2f)); \
    p = FMA(p, z, C(0.1333296820144401f));             \
    p = FMA(p, z, C(-0.33333331952545429f));

__device__ __forceinline__ float tanh_small(float y)
{
    const float z = y * y;
    float p;
    KV_TANH_POLY(fmaf, f1, z, p)
    return fmaf(y * z, p, y);
}

// g(t_p + s) - g(t_p) to about 1e-3 in absolute terms, for the range check (whose window is 12
// wide): the same form with e^{+-s} from ex2.approx and phi(+-s) = e^{+-s} - 1 -+ s directly
// (no series), with e^{-2vt} and e^{+-s} returned for the slope.
__device__ __forceinline__ float delta_g_coarse(const BinsF& b, float s, float& e2, float& es,
                                                float& ems)
{
    es = ex2_approx(s * LOG2E_F);
    ems = rcp_approx(es);
    const float vt = fmaf(b.v, s, b.u);
    e2 = ex2_approx(-2.0f * LOG2E_F * vt);
    const float d = fmaf(lg2_approx(1.0f + e2), LN2_F, -b.lu);
    const float php = (es - 1.0f) - s, phm = (ems - 1.0f) + s;
    return fmaf(b.c1, s, d) - fmaf(b.ap, php, b.am * phm);
}

// d/ds of delta_g_coarse at the same s, from the values it returned: g'(t_p + s) written as
// (v - x sinh t_p) - 2v e^{-2vt} / (1 + e^{-2vt}) - (x e^{t_p}/2)(e^s - 1) + (x e^{-t_p}/2)(e^{-s} - 1).
__device__ __forceinline__ float delta_g_slope_f32(const BinsF& b, float e2, float es, float ems)
{
    float dl = -2.0f * b.v * e2 * rcp_approx(1.0f + e2);
    return b.c1 + dl - b.ap * (es - 1.0f) + b.am * (ems - 1.0f);
}

// delta_g_coarse and delta_g_slope_f32 at two points at once (paired instructions; the
// exponentials per component).
__device__ __forceinline__ float2 delta_g_coarse2(const BinsF& b, float2 s, float2& e2, float2& es,
                                                  float2& ems)
{
    const float2 el = mul2(s, f2(LOG2E_F));
    es = make_float2(ex2_approx(el.x), ex2_approx(el.y));
    ems = make_float2(rcp_approx(es.x), rcp_approx(es.y));
    const float2 ea = mul2(fma2(f2(b.v), s, f2(b.u)), f2(-2.0f * LOG2E_F));
    e2 = make_float2(ex2_approx(ea.x), ex2_approx(ea.y));
    const float2 ope = add2(f2(1.0f), e2);
    const float2 d = fma2(make_float2(lg2_approx(ope.x), lg2_approx(ope.y)), f2(LN2_F), f2(-b.lu));
    const float2 php = fma2(s, f2(-1.0f), add2(es, f2(-1.0f)));  // (e^s - 1) - s
    const float2 phm = add2(add2(ems, f2(-1.0f)), s);            // (e^-s - 1) + s
    return fma2(f2(-b.ap), php, fma2(f2(-b.am), phm, fma2(f2(b.c1), s, d)));
}

__device__ __forceinline__ float2 delta_g_slope2(const BinsF& b, float2 e2, float2 es, float2 ems)
{
    const float2 ope = add2(f2(1.0f), e2);
    const float2 dl = mul2(mul2(f2(-2.0f * b.v), e2), make_float2(rcp_approx(ope.x), rcp_approx(ope.y)));
    return fma2(f2(-b.ap), add2(es, f2(-1.0f)), fma2(f2(b.am), add2(ems, f2(-1.0f)), add2(f2(b.c1), dl)));
}

// The bin constants rescaled once per pair so that a bin works in base-2 exponent units.  The
// weight is split as
//   e^{g(t) - g(t_p)} = e^{-lu} (1 + e^{-2vt}) 2^{c1 s + N(s)},   lu = log1p(e^{-2u}),
// with c1 = (v - x sinh t_p) log2 e and N(s) = -((x e^{t_p}/2) phi(s) + (x e^{-t_p}/2) phi(-s)) log2 e,
// so that log1p(e^{-2vt}) is never taken (its exponential is the factor 1 + e^{-2vt}) and the
// tanh integrand needs no reciprocal: w tanh(vt) = e^{-lu} (1 - e^{-2vt}) 2^{c1 s + N(s)}.
struct BinsK {
    float c1, ap, am, lu;  // v - x sinh t_p, x e^{+-t_p}/2, log1p(e^{-2u}), each times log2 e
    float hep, hem;        // e^{+-t_p} / 2
    float cA, cB;          // x cosh t_p, x sinh t_p, times log2 e
    float nA, nB;          // -cA, -cB
    float nap, nam;        // -ap, -am
    float nv2, nu2;        // -2 v log2 e, -2 u log2 e: e^{-2vt} = 2^{nv2 s + nu2}
    float kc;              // e^{-lu} = 1 / (1 + e^{-2u})
    float s2;              // -1 / (x log2 e) = -cosh t_p / cA: turns sum w nxc into sum w cosh t
};

__device__ __forceinline__ BinsK bins_k(const BinsF& b)
{
    BinsK k;
    k.c1 = b.c1 * LOG2E_F;
    k.ap = b.ap * LOG2E_F;
    k.am = b.am * LOG2E_F;
    k.lu = b.lu * LOG2E_F;
    k.hep = 0.5f * b.ep;
    k.hem = 0.5f * b.em;
    k.cA = b.xch * LOG2E_F;
    k.cB = b.xsh * LOG2E_F;
    k.nA = -k.cA;
    k.nB = -k.cB;
    k.nap = -k.ap;
    k.nam = -k.am;
    k.nv2 = -2.0f * LOG2E_F * b.v;
    k.nu2 = -2.0f * LOG2E_F * b.u;
    k.kc = ex2_approx(-k.lu);  // e^{-lu} from the same lu as the offset g(t_p), which it cancels
    k.s2 = -(k.hep + k.hem) * rcp_approx(k.cA);
    return k;
}

// N(s) for two bins:
//   |s| <= 1: phi(+-s) = z (E(z) +- s O(z)), so N = -z (x cosh t_p E + x sinh t_p s O);
//   |s| > 1:  N = x cosh t_p + x sinh t_p s - x cosh t  with  x cosh t = (x e^{t_p}/2) e^s + (x e^{-t_p}/2) e^{-s}
// (all times log2 e).  With DERIV, nxc = -(x cosh t) log2 e is returned for the d/dx integrand
// (w cosh t = w nxc times -1/(x log2 e), applied once to the sum), so that the cosh t of the
// integrand and the exponent share their products.
template <bool DERIV>
__device__ __forceinline__ float2 x_part2(const BinsK& k, float2 s, float2& nxc)
{
    const float2 z = mul2(s, s);
    float2 E, O;
    KV_PHI_SERIES(mul2, fma2, f2, z, E, O)
    const float2 so = mul2(s, O);
    const float2 ns = mul2(z, fma2(f2(k.nA), E, mul2(f2(k.nB), so)));
    const float2 el = mul2(s, f2(LOG2E_F));
    const float2 es = make_float2(ex2_approx(el.x), ex2_approx(el.y));
    const float2 ems = make_float2(rcp_approx(es.x), rcp_approx(es.y));
    float2 nl;
    if constexpr (DERIV) {
        nxc = fma2(f2(k.nap), es, mul2(f2(k.nam), ems));
        nl = add2(fma2(f2(k.cB), s, f2(k.cA)), nxc);
    } else {
        nl = fma2(f2(k.nap), es, fma2(f2(k.nam), ems, fma2(f2(k.cB), s, f2(k.cA))));
    }
    return make_float2(fabsf(s.x) <= PHI_SERIES_MAX ? ns.x : nl.x, fabsf(s.y) <= PHI_SERIES_MAX ? ns.y : nl.y);
}

template <bool DERIV>
__device__ __forceinline__ float x_part(const BinsK& k, float s, float& nxc)
{
    const float z = s * s;
    float E, O;
    KV_PHI_SERIES(__fmul_rn, fmaf, f1, z, E, O)
    const float ns = z * fmaf(k.nA, E, k.nB * (s * O));
    const float es = ex2_approx(s * LOG2E_F);
    const float ems = rcp_approx(es);
    float nl;
    if constexpr (DERIV) {
        nxc = fmaf(k.nap, es, k.nam * ems);
        nl = fmaf(k.cB, s, k.cA) + nxc;
    } else {
        nl = fmaf(k.nap, es, fmaf(k.nam, ems, fmaf(k.cB, s, k.cA)));
    }
    return fabsf(s) <= PHI_SERIES_MAX ? ns : nl;
}

// vt below this uses tanh_small; in the bins the test is on -2 vt log2 e (EA_SERIES_MIN)
constexpr float TANH_SERIES_MAX = 0.35f;
constexpr float EA_SERIES_MIN = -2.0f * LOG2E_F * TANH_SERIES_MAX;

// One FP32 bin at m = mf (a float holding a small integer, exact): its weight c e^{g(t_m) - g(t_p)}
// and the two derivative integrands' weights, all divided by e^{-lu} (the sums apply that factor
// once): wp = c 2^{c1 s + N(s)}, w = wp (1 + e^{-2vt}) and w tanh(vt) = wp (1 - e^{-2vt}), the
// latter as one fused multiply-add (the product rounded once).  `c` is the trapezoid factor
// (1/2 at the ends, else 1).  With VOTE (all 32 lanes of the warp run the same bins together)
// the series for tanh(vt) is evaluated only when some lane of the warp needs it.
template <bool DERIV, bool VOTE>
__device__ __forceinline__ void bin_f32(const BinsF& b, const BinsK& k, float mf, float c, float& w,
                                        float& w1, float& w2)
{
    const float s = fmaf(mf, b.h, b.s0);
    float nxc;
    const float N = x_part<DERIV>(k, s, nxc);
    const float ea = fmaf(k.nv2, s, k.nu2);
    const float e2 = ex2_approx(ea);  // e^{-2vt}
    const float wp = c * ex2_approx(fmaf(k.c1, s, N));
    w = fmaf(wp, e2, wp);
    if (DERIV) {
        const float t = b.tp + s;
        float d = fmaf(wp, -e2, wp);  // w tanh(vt)
        const bool small = ea > EA_SERIES_MIN;
        if (!VOTE || __any_sync(0xffffffffu, small))
            d = small ? w * tanh_small(ea * (-0.5f * LN2_F)) : d;
        w1 = t * d;
        w2 = w * nxc;  // w cosh t times -x log2 e
    }
}

// ------------------------------------------------------------------ two bins per instruction

__device__ __forceinline__ float2 tanh_small2(float2 y)
{
    const float2 z = mul2(y, y);
    float2 p;
    KV_TANH_POLY(fma2, f2, z, p)
    return fma2(mul2(y, z), p, y);
}

// bin_f32 for the two bins m = mf.x and mf.y; with CK their trapezoid factors are c.x and c.y,
// without they are 1 (no multiplication).
template <bool DERIV, bool VOTE, bool CK>
__device__ __forceinline__ void bin_f32x2(const BinsF& b, const BinsK& k, float2 mf, float2 c, float2& w,
                                          float2& w1, float2& w2)
{
    const float2 s = fma2(mf, f2(b.h), f2(b.s0));
    float2 nxc;
    const float2 N = x_part2<DERIV>(k, s, nxc);
    const float2 ea = fma2(f2(k.nv2), s, f2(k.nu2));
    const float2 e2 = make_float2(ex2_approx(ea.x), ex2_approx(ea.y));  // e^{-2vt}
    const float2 dg = fma2(f2(k.c1), s, N);
    float2 wp = make_float2(ex2_approx(dg.x), ex2_approx(dg.y));
    if constexpr (CK) wp = mul2(c, wp);
    w = fma2(wp, e2, wp);
    if (DERIV) {
        const float2 t = add2(f2(b.tp), s);
        float2 d = fma2(wp, make_float2(-e2.x, -e2.y), wp);  // w tanh(vt)
        const bool kx = ea.x > EA_SERIES_MIN, ky = ea.y > EA_SERIES_MIN;
        if (!VOTE || __any_sync(0xffffffffu, kx || ky)) {
            const float2 wt = mul2(w, tanh_small2(mul2(ea, f2(-0.5f * LN2_F))));  // vt from ea
            d = make_float2(kx ? wt.x : d.x, ky ? wt.y : d.y);
        }
        w1 = mul2(t, d);
        w2 = mul2(w, nxc);  // w cosh t times -x log2 e
    }
}

// The three sums over bins m = lane, lane + L, ... <= n: each block of four bins is added
// pairwise (two rounding levels); the block sums are compensated (Kahan, COMP; with L = 1 the sums
// of two consecutive blocks are added first and compensated together, one Kahan step per eight
// bins), so that the relative error stays a few units of 2^-24 for any bin count, or added
// plainly (!COMP: 1 addition per term), which for all-positive terms bounds the relative error by
// (2 + k) units of 2^-24 after k sequential additions — at most 13 units for up to 40 bins per
// lane (10 blocks and one tail bin), 7.7e-7, so that a ratio of two sums stays within 1.6e-6.
// The end weight 1/2 of bin 0 is applied to the first block's first term (lane 0 only); bin n
// falls in the tail loop, which selects its weight, unless the caller already has its terms
// (with_end, L = 1 only: e0, e1, e2 are bin n's contributions to the three sums, which then start
// from them).  VOTE requires L = 1 and all 32 lanes of the warp in the call with the same n.
constexpr int kPlainSumsMaxBins = 40;

template <int L, bool DERIV, bool VOTE = false, bool COMP = true>
__device__ __forceinline__ void sums_f32(const BinsF& b, int lane, float& S0, float& S1, float& S2,
                                         bool with_end = false, float e0 = 0.0f, float e1 = 0.0f,
                                         float e2 = 0.0f)
{
    const BinsK k = bins_k(b);
    KahanSum<float> k0, k1, k2;
    k0.init();
    k1.init();
    k2.init();
    // the bins' terms leave out the factor e^{-lu} = 1 / (1 + e^{-2u}), applied to the sums at
    // the end; bin n's terms from the caller include it
    if (with_end) {
        const float rkc = 1.0f + b.e2u;
        k0.s = e0 * rkc;
        k1.s = e1 * rkc;
        k2.s = e2 * rkc;
    }
    float q0 = k0.s, q1 = k1.s, q2 = k2.s;  // plain block sums (COMP = false)
    const int last = with_end ? b.n - 1 : b.n;
    int m = lane;
    float mf = (float)lane;
    // the first block carries bin 0's factor 1/2 (lane 0); the later ones multiply by nothing
    auto block = [&](auto ck) {
        constexpr bool CK = decltype(ck)::value;
        float2 wa, w1a, w2a, wb, w1b, w2b;
        bin_f32x2<DERIV, VOTE, CK>(b, k, make_float2(mf, mf + (float)L), make_float2(lane == 0 ? 0.5f : 1.0f, 1.0f),
                                   wa, w1a, w2a);
        bin_f32x2<DERIV, VOTE, false>(b, k, make_float2(mf + (float)(2 * L), mf + (float)(3 * L)), f2(1.0f), wb, w1b, w2b);
        const float2 p0 = add2(wa, wb);
        if (COMP) k0.add(p0.x + p0.y); else q0 += p0.x + p0.y;
        if (DERIV) {
            const float2 p1 = add2(w1a, w1b), p2 = add2(w2a, w2b);
            if (COMP) {
                k1.add(p1.x + p1.y);
                k2.add(p2.x + p2.y);
            } else {
                q1 += p1.x + p1.y;
                q2 += p2.x + p2.y;
            }
        }
    };
    if (m + 3 * L < b.n) {
        block(std::true_type());
        m += 4 * L;
        mf += (float)(4 * L);
    }
    if constexpr (COMP && L == 1) {
        // two blocks per trip: their block sums are added (one more rounding level) and take one
        // Kahan step together (1.1 FP32 operations per bin fewer than a step per block)
        float2 wa, w1a, w2a, wb, w1b, w2b;
        for (; m + 7 < b.n; m += 8, mf += 8.0f) {
            bin_f32x2<DERIV, VOTE, false>(b, k, make_float2(mf, mf + 1.0f), f2(1.0f), wa, w1a, w2a);
            bin_f32x2<DERIV, VOTE, false>(b, k, make_float2(mf + 2.0f, mf + 3.0f), f2(1.0f), wb, w1b, w2b);
            const float2 p0 = add2(wa, wb);
            float2 p1, p2;
            if (DERIV) {
                p1 = add2(w1a, w1b);
                p2 = add2(w2a, w2b);
            }
            const float r0 = p0.x + p0.y;
            const float r1 = DERIV ? p1.x + p1.y : 0.0f, r2 = DERIV ? p2.x + p2.y : 0.0f;
            bin_f32x2<DERIV, VOTE, false>(b, k, make_float2(mf + 4.0f, mf + 5.0f), f2(1.0f), wa, w1a, w2a);
            bin_f32x2<DERIV, VOTE, false>(b, k, make_float2(mf + 6.0f, mf + 7.0f), f2(1.0f), wb, w1b, w2b);
            const float2 q0 = add2(wa, wb);
            k0.add(r0 + (q0.x + q0.y));
            if (DERIV) {
                const float2 q1 = add2(w1a, w1b), q2 = add2(w2a, w2b);
                k1.add(r1 + (q1.x + q1.y));
                k2.add(r2 + (q2.x + q2.y));
            }
        }
    }
    for (; m + 3 * L < b.n; m += 4 * L, mf += (float)(4 * L)) block(std::false_type());
    for (; m <= last; m += L, mf += (float)L) {
        float w, w1, w2;
        bin_f32<DERIV, VOTE>(b, k, mf, (m == 0 || m == b.n) ? 0.5f : 1.0f, w, w1, w2);
        if (COMP) k0.add(w); else q0 += w;
        if (DERIV) {
            if (COMP) {
                k1.add(w1);
                k2.add(w2);
            } else {
                q1 += w1;
                q2 += w2;
            }
        }
    }
    if (!COMP) {
        k0.s = q0;
        k1.s = q1;
        k2.s = q2;
    }
    S0 = lane_sum<float, L>(k0.value()) * k.kc;
    S1 = DERIV ? lane_sum<float, L>(k1.value()) * k.kc : 0.0f;
    S2 = DERIV ? lane_sum<float, L>(k2.value()) * (k.s2 * k.kc) : 0.0f;
}

// ------------------------------------------------------------------ second derivatives
// Sec. 4.1 with n + m = 2: K_vv, K_vx, K_xx integrate t^2 cosh(vt), -t cosh(t) sinh(vt) and
// cosh^2(t) cosh(vt) times e^{-x cosh t} over the same bins.  With weights w ~ cosh(vt) e^{-x cosh t},
// a = t tanh(vt) and c = cosh t, the log-derivatives are moments:
//   d/dv log K = E[a],  d/dx log K = -E[c],
//   d2/dv2 log K = E[t^2 sech^2(vt)] + Var(a),  d2/dv dx log K = -Cov(a, c),  d2/dx2 log K = Var(c).
// The plain forms E[t^2] - E[a]^2 etc. cancel badly where the range is narrow (d2/dx2 ~ 1/(2x^2)
// at large x against E[c]^2 ~ 1), so the sums run over the shifts about the reference point,
// da = a - t_p tanh(u) and dc = cosh t - cosh t_p, each formed without cancellation:
//   da = s tanh(vt) - t_p 2 (e^{-2vt} - e^{-2u}) / ((1 + e^{-2vt})(1 + e^{-2u})),
//        with e^{-2vt} - e^{-2u} = e^{-2u} expm1(-2vs) where |2vs| < 1/2 (else the plain difference,
//        which does not cancel there and does not turn 0 * inf into NaN when e^{-2u} underflows)
//   dc = sinh(t_p) s + (e^{t_p}/2) phi(s) + (e^{-t_p}/2) phi(-s)   (= 2 sinh((t+t_p)/2) sinh(s/2))
// and Var(a) = E[da^2] - E[da]^2 etc., where E[da], E[dc] are small near the peak.
template <typename T>
struct Sums2 {
    T s0, a1, a2, c1, c2, x, q;  // sum w, w da, w da^2, w dc, w dc^2, w da dc, w t^2 sech^2(vt)
};

// First and second log-derivatives from the sums, with a_r = t_p tanh(u), c_r = cosh t_p (for
// |v|; the caller applies the sign of v to dv and dvx).
template <typename T>
__device__ __forceinline__ void moments_finish(const Sums2<T>& m, T ar, T cr, T& dv, T& dx, T& d2v,
                                               T& dvx, T& d2x)
{
    const T r = T(1) / m.s0;
    const T ea = m.a1 * r, ec = m.c1 * r;
    dv = ar + ea;
    dx = -(cr + ec);
    d2v = m.q * r + (m.a2 * r - ea * ea);
    d2x = m.c2 * r - ec * ec;
    dvx = ea * ec - m.x * r;
}

template <typename T, int L>
__device__ __forceinline__ Sums2<T> lane_sums2(const KahanSum<T> (&k)[7])
{
    Sums2<T> m;
    m.s0 = lane_sum<T, L>(k[0].value());
    m.a1 = lane_sum<T, L>(k[1].value());
    m.a2 = lane_sum<T, L>(k[2].value());
    m.c1 = lane_sum<T, L>(k[3].value());
    m.c2 = lane_sum<T, L>(k[4].value());
    m.x = lane_sum<T, L>(k[5].value());
    m.q = lane_sum<T, L>(k[6].value());
    return m;
}

// The seven sums in FP64 with the first-derivative bins' scheme (sums_f64): the weight as
// (1 + e^{-2vt})/(1 + e^{-2u}) exp(c1 s + N(s)), phi(+-s) from the minimax polynomials for |s| <= 1
// and from e^{+-s} beyond, e^{+-s} and e^{-2vt} by recurrence with an exact refresh every
// kRefreshF64 steps, sums plain within a block and compensated across blocks; dc = cosh t -
// cosh t_p = sinh t_p s + (e^{t_p} phi(s) + e^{-t_p} phi(-s))/2 from the same phi values, and
// e^{-2vt} - e^{-2u} = e^{-2u} expm1(-2vs) where |2vs| < 1/2.
template <int L>
__device__ Sums2<double> sums2_f64(const BinsD& b, int lane)
{
    KahanSum<double> k[7];
    double q[7];
    for (int j = 0; j < 7; ++j) {
        k[j].init();
        q[j] = 0.0;
    }
    const double kc = 1.0 / (1.0 + b.e2u);
    const double ap = 0.5 * b.x * b.ep, am = 0.5 * b.x * b.em;
    const double step = L * b.h;
    const double qs = exp(step), qsi = exp(-step), q2 = exp(-2.0 * b.v * step);
    double es = 1.0, esi = 1.0, e2 = 1.0;
    int since = kRefreshF64;
    for (int m = lane; m <= b.n; m += L) {
        const double s = fma((double)m, b.h, b.s0);
        const double t = b.tp + s;
        if (since == kRefreshF64) {
            es = exp(s);
            esi = 1.0 / es;
            e2 = exp(-2.0 * b.v * t);
            since = 0;
            for (int j = 0; j < 7; ++j) {
                k[j].add(q[j]);
                q[j] = 0.0;
            }
        }
        const double z = s * s;
        double E, O;
        phi_parts_f64(z, E, O);
        const bool small = fabs(s) <= 1.0;
        const double so = s * O;
        const double php = small ? z * (E + so) : (es - 1.0) - s;   // phi(s)
        const double phm = small ? z * (E - so) : (esi - 1.0) + s;  // phi(-s)
        const double N = -fma(ap, php, am * phm);
        const double dc = fma(b.shp, s, 0.5 * fma(b.ep, php, b.em * phm));
        const double c = (m == 0 || m == b.n) ? 0.5 : 1.0;
        const double ope = 1.0 + e2;
        const double w = c * kc * ope * exp(fma(b.c1, s, N));
        const double r = 1.0 / ope;
        const double vt = b.v * t;
        double qt = 1.0 - e2;  // (1 + e^{-2vt}) tanh(vt)
        if (vt < 0.5) qt = -expm1(-2.0 * vt);
        const double th = qt * r;
        const double vs2 = -2.0 * b.v * s;
        double de = e2 - b.e2u;  // e^{-2vt} - e^{-2u}
        if (fabs(vs2) < 0.5) de = b.e2u * expm1(vs2);
        const double da = s * th - b.tp * 2.0 * de * r * kc;
        const double wda = w * da, wdc = w * dc;
        q[0] += w;
        q[1] += wda;
        q[2] = fma(wda, da, q[2]);
        q[3] += wdc;
        q[4] = fma(wdc, dc, q[4]);
        q[5] = fma(wda, dc, q[5]);
        q[6] = fma(w * (t * t), 4.0 * e2 * r * r, q[6]);
        es *= qs;
        esi *= qsi;
        e2 *= q2;
        ++since;
    }
    for (int j = 0; j < 7; ++j) k[j].add(q[j]);
    return lane_sums2<double, L>(k);
}

// expm1(y) for |y| < 1/2 (two values): y (1 + y/2 + ... + y^7/8!), relative error about 1e-8
// before rounding.
__device__ __forceinline__ float2 expm1_small2(float2 y)
{
    float2 p = f2(1.0f / 40320.0f);
    p = fma2(p, y, f2(1.0f / 5040.0f));
    p = fma2(p, y, f2(1.0f / 720.0f));
    p = fma2(p, y, f2(1.0f / 120.0f));
    p = fma2(p, y, f2(1.0f / 24.0f));
    p = fma2(p, y, f2(1.0f / 6.0f));
    p = fma2(p, y, f2(0.5f));
    return fma2(mul2(y, y), p, y);
}

// Bins per block of the FP32 second-derivative sums: plain sums within a block, compensated
// (Kahan) across blocks.
constexpr int kBlockSums2 = 8;

// Two bins (the components of s) of the seven sums, in paired FP32 instructions, added to acc:
// the fast path's weight split w = (1 + e^{-2vt}) 2^{c1 s + N(s) + cl} without the per-pair factor
// e^{-lu} (every sum carries it, so the moments do not see it; sums2_f32 applies it to S0), cl the
// trapezoid factor's log2 (-1 at the end bins, else 0); 1/(1 + e^{-2vt}) from the approximate
// reciprocal, tanh(vt) from its polynomial below vt = 0.35, e^{-2vt} - e^{-2u} as
// e^{-2u} expm1(-2vs) from a polynomial where |2vs| < 1/2, and
// dc = cosh t - cosh t_p = sinh t_p s + (e^{t_p} phi(s) + e^{-t_p} phi(-s))/2; acc[6] is the sum
// of w t^2 sech^2(vt) / 4.  With VOTE (all 32 lanes of the warp in the call) the two polynomials
// are evaluated only when some lane of the warp needs them.
template <bool VOTE>
__device__ __forceinline__ void sums2_bins2(const BinsF& b, const BinsK& kk, float2 s, float2 cl,
                                            float (&acc)[7])
{
    const float2 z = mul2(s, s);
    float2 E, O;
    KV_PHI_SERIES(mul2, fma2, f2, z, E, O)
    const float2 so = mul2(s, O);
    const float2 pp = mul2(z, add2(E, so)), pm = mul2(z, sub2(E, so));
    const float2 el = mul2(s, f2(LOG2E_F));
    const float2 es = make_float2(ex2_approx(el.x), ex2_approx(el.y));
    const float2 ems = make_float2(rcp_approx(es.x), rcp_approx(es.y));
    const float2 pl = sub2(add2(es, f2(-1.0f)), s), ml = add2(add2(ems, f2(-1.0f)), s);
    const bool sx = fabsf(s.x) <= PHI_SERIES_MAX, sy = fabsf(s.y) <= PHI_SERIES_MAX;
    const float2 php = make_float2(sx ? pp.x : pl.x, sy ? pp.y : pl.y);  // phi(s)
    const float2 phm = make_float2(sx ? pm.x : ml.x, sy ? pm.y : ml.y);  // phi(-s)
    const float2 ea = fma2(f2(kk.nv2), s, f2(kk.nu2));
    const float2 e2 = make_float2(ex2_approx(ea.x), ex2_approx(ea.y));  // e^{-2vt}
    const float2 ope = add2(f2(1.0f), e2);
    const float2 rope = make_float2(rcp_approx(ope.x), rcp_approx(ope.y));
    const float2 dg = fma2(f2(kk.c1), s, fma2(f2(kk.nap), php, fma2(f2(kk.nam), phm, cl)));
    const float2 w = mul2(ope, make_float2(ex2_approx(dg.x), ex2_approx(dg.y)));
    const float2 vt = fma2(f2(b.v), s, f2(b.u));
    float2 th = mul2(sub2(f2(1.0f), e2), rope);
    {
        const bool kx = vt.x < TANH_SERIES_MAX, ky = vt.y < TANH_SERIES_MAX;
        if (!VOTE || __any_sync(0xffffffffu, kx || ky)) {
            const float2 ts = tanh_small2(vt);
            th = make_float2(kx ? ts.x : th.x, ky ? ts.y : th.y);
        }
    }
    const float2 t = add2(f2(b.tp), s);
    const float2 vs2 = mul2(f2(-2.0f * b.v), s);
    float2 de = sub2(e2, f2(b.e2u));
    {
        const bool kx = fabsf(vs2.x) < 0.5f, ky = fabsf(vs2.y) < 0.5f;
        if (!VOTE || __any_sync(0xffffffffu, kx || ky)) {
            const float2 des = mul2(f2(b.e2u), expm1_small2(vs2));
            de = make_float2(kx ? des.x : de.x, ky ? des.y : de.y);
        }
    }
    const float2 da = fma2(s, th, mul2(f2(-2.0f * b.tp * kk.kc), mul2(de, rope)));
    const float2 dc = fma2(f2(b.shp), s, fma2(f2(kk.hep), php, mul2(f2(kk.hem), phm)));
    const float2 wda = mul2(w, da), wdc = mul2(w, dc);
    const float2 wq = mul2(mul2(w, mul2(t, t)), mul2(e2, mul2(rope, rope)));  // w t^2 sech^2(vt) / 4
    acc[0] += w.x + w.y;
    acc[1] += wda.x + wda.y;
    acc[2] = fmaf(wda.x, da.x, fmaf(wda.y, da.y, acc[2]));
    acc[3] += wdc.x + wdc.y;
    acc[4] = fmaf(wdc.x, dc.x, fmaf(wdc.y, dc.y, acc[4]));
    acc[5] = fmaf(wda.x, dc.x, fmaf(wda.y, dc.y, acc[5]));
    acc[6] += wq.x + wq.y;
}

template <int L, bool VOTE = false>
__device__ Sums2<float> sums2_f32(const BinsF& b, int lane)
{
    const BinsK kk = bins_k(b);
    KahanSum<float> k[7];
    float acc[7];
    for (int j = 0; j < 7; ++j) {
        k[j].init();
        acc[j] = 0.0f;
    }
    int in_block = 0;
    int m = lane;
    float mf = (float)lane;
    for (; m + L <= b.n; m += 2 * L, mf += (float)(2 * L)) {
        const float2 s = fma2(make_float2(mf, mf + (float)L), f2(b.h), f2(b.s0));
        const float2 cl = make_float2(m == 0 ? -1.0f : 0.0f, m + L == b.n ? -1.0f : 0.0f);
        sums2_bins2<VOTE>(b, kk, s, cl, acc);
        in_block += 2;
        if (in_block == kBlockSums2) {
            for (int j = 0; j < 7; ++j) {
                k[j].add(acc[j]);
                acc[j] = 0.0f;
            }
            in_block = 0;
        }
    }
    if (m <= b.n) {
        // the one bin left (the second component's weight is zeroed through its exponent)
        const float s = fmaf(mf, b.h, b.s0);
        sums2_bins2<VOTE>(b, kk, f2(s), make_float2((m == 0 || m == b.n) ? -1.0f : 0.0f, -INFINITY), acc);
    }
    for (int j = 0; j < 7; ++j) k[j].add(acc[j]);
    // the factor e^{-lu} the bins left out, and sech^2(vt) = 4 e^{-2vt} / (1 + e^{-2vt})^2
    Sums2<float> r = lane_sums2<float, L>(k);
    r.s0 *= kk.kc;
    r.a1 *= kk.kc;
    r.a2 *= kk.kc;
    r.c1 *= kk.kc;
    r.c2 *= kk.kc;
    r.x *= kk.kc;
    r.q *= 4.0f * kk.kc;
    return r;
}

}  // namespace kvd
