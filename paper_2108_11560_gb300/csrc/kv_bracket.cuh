// FP64 range finding for one (v, x) pair: Sec. 2.1-2.3 and Algorithms 1-3.
//
// g(t) = log cosh(vt) - x cosh t is unimodal on t >= 0 (g''' <= 0, Sec. 2.1).  The peak t_p is
// the zero of g' (Algorithm 1 brackets it by doubling, Algorithm 2 refines it by bisection with a
// clipped Newton step); the ends t0 <= t_p <= t1 are the zeros of h = g - g(t_p) - log eps.
//
// Conventions (the paper's pseudocode is garbled in places; these readings are the library's):
//  * FindZero(F, t_neg, t_pos): t_neg is where F < 0, t_pos where F >= 0.  Each iteration takes
//    the bisection point and the Newton point from the current negative end, clipped to the
//    closed interval between the ORIGINAL negative end and the bisection point (a non-finite
//    Newton point becomes the bisection point); it returns the negative end after exactly
//    max_iter iterations, so every thread runs the same trip count.
//  * FindRange(F, t0): doubles 2^m from m = 0 while F(t0 + 2^{m+1}) >= 0, at most KV_RANGE_CAP
//    times; if it stops at m = 0 and F(t0 + 1) < 0, the positive end is t0 itself.
//  * Function values are cached across iterations: every point is evaluated once, together with
//    its derivative, which changes no result.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace kvd {

constexpr int KV_RANGE_CAP = 11;  // t up to 2^12 above the start: every finite double input
constexpr double LN2_D = 0.693147180559945309417232121458176568;

// log cosh(a) for a >= 0 without overflow: a + log(1 + e^{-2a}) - log 2.
__device__ __forceinline__ double log_cosh_d(double a) { return a + log1p(exp(-2.0 * a)) - LN2_D; }

struct PairD {
    double v, x;     // |v| and x
    double G;        // g(t_p)
    double log_eps;  // log of the range's eps
};

// 1/(1 + e2) and 1/et from one division: q = 1/((1 + e2) et), then et q and (1 + e2) q (two
// divisions where the product overflows, which only a capped doubling search far out reaches).
__device__ __forceinline__ void two_reciprocals(double ope, double et, double& r, double& eti)
{
    const double d = ope * et;
    if (d < INFINITY) {
        const double q = 1.0 / d;
        r = et * q;
        eti = ope * q;
    } else {
        r = 1.0 / ope;
        eti = 1.0 / et;
    }
}

// g'(t) and g''(t) at t >= 0 (Sec. 2.1), sharing e^{-2vt} and e^t.
__device__ __forceinline__ void eval_g1_g2(const PairD& p, double t, double& g1, double& g2)
{
    double e2 = exp(-2.0 * p.v * t);
    double et = exp(t);
    double r, eti;
    two_reciprocals(1.0 + e2, et, r, eti);
    double th = (1.0 - e2) * r;      // tanh(vt)
    double sech2 = 4.0 * e2 * r * r; // sech^2(vt)
    g1 = p.v * th - p.x * 0.5 * (et - eti);
    g2 = p.v * p.v * sech2 - p.x * 0.5 * (et + eti);
}

// h(t) = g(t) - G - log eps and h'(t) = g'(t) at t >= 0.
__device__ __forceinline__ void eval_h_h1(const PairD& p, double t, double& h, double& h1)
{
    double a = p.v * t;
    double e2 = exp(-2.0 * a);
    double et = exp(t);
    double r, eti;
    two_reciprocals(1.0 + e2, et, r, eti);
    double th = (1.0 - e2) * r;
    double g = a + log1p(e2) - LN2_D - p.x * 0.5 * (et + eti);
    h = g - p.G - p.log_eps;
    h1 = p.v * th - p.x * 0.5 * (et - eti);
}

// F and F' for the two searches: KIND 0 -> (g', g''), KIND 1 -> (h, g').
template <int KIND>
__device__ __forceinline__ void eval_F(const PairD& p, double t, double& F, double& dF)
{
    if (KIND == 0) eval_g1_g2(p, t, F, dF);
    else eval_h_h1(p, t, F, dF);
}

// Algorithm 1.  On return (t_pos, t_neg) bracket the zero; F_neg/dF_neg are F, F' at t_neg.
template <int KIND>
__device__ __forceinline__ bool find_range(const PairD& p, double t0, double& t_pos, double& t_neg,
                                           double& F_neg, double& dF_neg)
{
    int m = 0;
    double F, dF;
    eval_F<KIND>(p, t0 + 2.0, F, dF);
    while (m < KV_RANGE_CAP && F >= 0.0) {
        ++m;
        eval_F<KIND>(p, t0 + ldexp(1.0, m + 1), F, dF);
    }
    double lo = t0 + ldexp(1.0, m);
    if (m == 0) {
        double Flo, dFlo;
        eval_F<KIND>(p, lo, Flo, dFlo);
        if (!(Flo >= 0.0)) lo = t0;
    }
    t_pos = lo;
    t_neg = t0 + ldexp(1.0, m + 1);
    F_neg = F;
    dF_neg = dF;
    return F < 0.0;  // false only when the cap was hit before the sign changed
}

// Algorithm 2 with fixed max_iter.  Fa/dFa are F, F' at t_neg on entry.
template <int KIND>
__device__ __forceinline__ double find_zero(const PairD& p, double t_neg, double t_pos, double Fa,
                                            double dFa, int max_iter)
{
    double a = t_neg, b = t_pos;
    for (int i = 0; i < max_iter; ++i) {
        double shrink = a + (b - a) * 0.5;
        double newton = a - Fa / dFa;
        if (!isfinite(newton)) newton = shrink;
        double lo = fmin(t_neg, shrink), hi = fmax(t_neg, shrink);
        newton = fmin(fmax(newton, lo), hi);
        double Fs, dFs;
        eval_F<KIND>(p, shrink, Fs, dFs);
        if (Fs < 0.0) {
            a = shrink;
            Fa = Fs;
            dFa = dFs;
        } else {
            double Fn, dFn;
            eval_F<KIND>(p, newton, Fn, dFn);
            if (Fn < 0.0) {
                a = newton;
                b = shrink;
                Fa = Fn;
                dFa = dFn;
            } else {
                b = newton;
            }
        }
    }
    return a;
}

struct BracketD {
    double t0, tp, t1, G;
    bool capped;  // a FindRange hit its cap
};

// Algorithm 3 up to the integration: the peak, the offset g(t_p) and the range [t0, t1].
// With analytic_start the peak search skips Algorithm 1's doublings and runs Algorithm 2 on the
// bracket [0, asinh(v/x)]: g'(0) = 0 is the non-negative end, and at t = asinh(v/x),
// x sinh t = v > v tanh(vt), so g' < 0 there (the end is nudged up by 2^-40 relative, and the
// doublings are taken after all if g' is not negative there in rounded arithmetic).  The peak
// then comes from ten iterations on a different interval, so it differs from Algorithms 1-2's
// within their convergence; the range searches are unchanged.
__device__ __forceinline__ BracketD bracket_f64(double v, double x, double log_eps, int max_iter,
                                                bool analytic_start = false)
{
    PairD p{v, x, 0.0, log_eps};
    BracketD r;
    r.capped = false;
    double tp = 0.0;
    if (v * v - x > 0.0) {  // g''(0) = v^2 - x > 0: a peak at t_p > 0 (Sec. 2.1)
        double ts = 0.0, te = 0.0, F = 0.0, dF = 0.0;
        bool have = false;
        if (analytic_start) {
            te = asinh(v / x) * (1.0 + 0x1.0p-40);
            eval_g1_g2(p, te, F, dF);
            have = F < 0.0 && isfinite(te);
        }
        if (!have) r.capped |= !find_range<0>(p, 0.0, ts, te, F, dF);
        tp = find_zero<0>(p, te, ts, F, dF, max_iter);
    }
    double e2 = exp(-2.0 * v * tp);
    double et = exp(tp);
    p.G = v * tp + log1p(e2) - LN2_D - x * 0.5 * (et + 1.0 / et);
    double t0 = 0.0;
    double g0 = log1p(1.0) - LN2_D - x;  // g(0)
    if (g0 - p.G <= log_eps) {
        double h0, h1;
        eval_h_h1(p, 0.0, h0, h1);
        t0 = find_zero<1>(p, 0.0, tp, h0, h1, max_iter);
    }
    double ts, te, F, dF;
    r.capped |= !find_range<1>(p, tp, ts, te, F, dF);
    double t1 = find_zero<1>(p, te, ts, F, dF, max_iter);
    r.t0 = t0;
    r.tp = tp;
    r.t1 = t1;
    r.G = p.G;
    return r;
}

// ------------------------------------------------------------------ a pair's bracket on L lanes
// The same searches with the L lanes of a warp group (lane mask gm, first lane g0, this lane l)
// evaluating several of their points at once: FindRange evaluates t0 + 2^j for L consecutive j
// per round, FindZero the bisection point (lane 0) and the Newton point (lane 1) of an iteration
// together.  The points, the values and every decision are those of the one-lane searches above
// (every lane of the group holds the same state), so the bracket is the same; what shrinks is
// the number of instructions the warp issues (GB300's FP64 unit costs the same per warp
// instruction whatever the number of active lanes).  Every lane of the group takes every branch
// together, so the group's shuffles always meet.

struct LaneGroup {
    unsigned mask;  // the group's lanes in the warp
    int first;      // its first lane
    int l;          // this lane's place in it
};

__device__ __forceinline__ double group_take(const LaneGroup& G, double a, int k)
{
    return __shfl_sync(G.mask, a, G.first + k);
}

// Algorithm 1 on L lanes: the first j >= 1 where F(t0 + 2^j) is not >= 0 gives m = j - 1 (at
// most KV_RANGE_CAP); F(t0 + 1) (j = 0) decides the positive end when m = 0.
template <int KIND, int L>
__device__ __forceinline__ bool find_range_group(const PairD& p, const LaneGroup& G, double t0, double& t_pos,
                                                 double& t_neg, double& F_neg, double& dF_neg)
{
    constexpr int JMAX = KV_RANGE_CAP + 1;
    int jneg = -1;  // the first j >= 1 with F not >= 0
    double F1 = 0.0, Fn = 0.0, dFn = 0.0;
    for (int r = 0; jneg < 0 && r * L <= JMAX; ++r) {
        const int j = r * L + G.l;
        double F = 0.0, dF = 0.0;
        if (j <= JMAX) eval_F<KIND>(p, t0 + ldexp(1.0, j), F, dF);
        if (r == 0) F1 = group_take(G, F, 0);  // F(t0 + 1)
        const bool stop = j >= 1 && j <= JMAX && !(F >= 0.0);
        const unsigned b = (__ballot_sync(G.mask, stop) & G.mask) >> G.first;
        const int k = b ? __ffs(b) - 1 : (JMAX - r * L < L - 1 ? JMAX - r * L : L - 1);
        Fn = group_take(G, F, k);
        dFn = group_take(G, dF, k);
        if (b) jneg = r * L + k;
    }
    const int m = jneg < 0 ? KV_RANGE_CAP : jneg - 1;
    double lo = t0 + ldexp(1.0, m);
    if (m == 0 && !(F1 >= 0.0)) lo = t0;
    t_pos = lo;
    t_neg = t0 + ldexp(1.0, m + 1);
    F_neg = Fn;
    dF_neg = dFn;
    return Fn < 0.0;
}

// Algorithm 2 on L >= 2 lanes: lane 1 evaluates the Newton point, the others the bisection point.
template <int KIND>
__device__ __forceinline__ double find_zero_group(const PairD& p, const LaneGroup& G, double t_neg, double t_pos,
                                                  double Fa, double dFa, int max_iter)
{
    double a = t_neg, b = t_pos;
    for (int i = 0; i < max_iter; ++i) {
        double shrink = a + (b - a) * 0.5;
        double newton = a - Fa / dFa;
        if (!isfinite(newton)) newton = shrink;
        double lo = fmin(t_neg, shrink), hi = fmax(t_neg, shrink);
        newton = fmin(fmax(newton, lo), hi);
        double F, dF;
        eval_F<KIND>(p, G.l == 1 ? newton : shrink, F, dF);
        const double Fs = group_take(G, F, 0), dFs = group_take(G, dF, 0);
        const double Fn = group_take(G, F, 1), dFn = group_take(G, dF, 1);
        if (Fs < 0.0) {
            a = shrink;
            Fa = Fs;
            dFa = dFs;
        } else if (Fn < 0.0) {
            a = newton;
            b = shrink;
            Fa = Fn;
            dFa = dFn;
        } else {
            b = newton;
        }
    }
    return a;
}

// bracket_f64 on the L >= 2 lanes of a group; every lane returns the same bracket.
template <int L>
__device__ __forceinline__ BracketD bracket_f64_group(const LaneGroup& G, double v, double x, double log_eps,
                                                      int max_iter, bool analytic_start = false)
{
    static_assert(L >= 2, "the group searches need two lanes");
    PairD p{v, x, 0.0, log_eps};
    BracketD r;
    r.capped = false;
    double tp = 0.0;
    if (v * v - x > 0.0) {
        double ts = 0.0, te = 0.0, F = 0.0, dF = 0.0;
        bool have = false;
        if (analytic_start) {
            te = asinh(v / x) * (1.0 + 0x1.0p-40);
            eval_g1_g2(p, te, F, dF);
            have = F < 0.0 && isfinite(te);
        }
        if (!have) r.capped |= !find_range_group<0, L>(p, G, 0.0, ts, te, F, dF);
        tp = find_zero_group<0>(p, G, te, ts, F, dF, max_iter);
    }
    double e2 = exp(-2.0 * v * tp);
    double et = exp(tp);
    p.G = v * tp + log1p(e2) - LN2_D - x * 0.5 * (et + 1.0 / et);
    double t0 = 0.0;
    double g0 = log1p(1.0) - LN2_D - x;  // g(0)
    if (g0 - p.G <= log_eps) {
        double h0, h1;
        eval_h_h1(p, 0.0, h0, h1);
        t0 = find_zero_group<1>(p, G, 0.0, tp, h0, h1, max_iter);
    }
    double ts, te, F, dF;
    r.capped |= !find_range_group<1, L>(p, G, tp, ts, te, F, dF);
    double t1 = find_zero_group<1>(p, G, te, ts, F, dF, max_iter);
    r.t0 = t0;
    r.tp = tp;
    r.t1 = t1;
    r.G = p.G;
    return r;
}

}  // namespace kvd
