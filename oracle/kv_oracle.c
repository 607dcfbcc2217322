/*
 * CPU oracle for batched log K_v(x) and its derivatives in v and x.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this file;
 * only the test suite, the smoke check and the bench's CPU-baseline leg use it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Two computations live here:
 *
 *   O1  The paper's fixed-bin integration method, step by step, in the paper's order:
 *       Sec. 2.1 (the integrand f = cosh(vt) exp(-x cosh t), g = log f and its t-derivatives),
 *       Algorithm 1 (FindRange), Algorithm 2 (FindZero), Sec. 2.3 (the range [t0, t1]),
 *       Sec. 2.4 Eq. (int) (trapezoid rule with c_0 = c_n = 1/2 in log-sum-exp form) and
 *       Algorithm 3 (LogBesselK).  The derivatives follow Sec. 4.1: the same bins carry the
 *       v-derivative integrand t sinh(vt) e^{-x cosh t} and the x-derivative integrand
 *       -cosh(t) cosh(vt) e^{-x cosh t}, each divided by the K sum.
 *       Second derivatives (Sec. 4.1, the integrands f^{(n,m)} with n + m = 2) come from the
 *       same bins: K_vv, K_vx, K_xx carry t^2 cosh(vt), -t cosh(t) sinh(vt) and cosh^2(t) cosh(vt)
 *       times e^{-x cosh t}, and the log-derivatives are their plain combinations
 *       d2/dv2 log K = K_vv/K - (K_v/K)^2 and likewise (reading R8).
 *       The file is compiled twice: with KV_REAL = double (the method in FP64, as the paper
 *       runs it) and with KV_REAL = long double (the same steps in wider arithmetic, used as the
 *       method's reference value at FP64 tolerances).  <tgmath.h> picks exp/expl etc. by type.
 *
 *   O2  (long double build only) The integral of Eq. (1)-(2) by dense adaptive Gauss-Legendre
 *       quadrature on a widened range found by a plain scan, independent of Algorithms 1-3.
 *       This is the truth that the method itself is measured against.
 *
 * Readings of passages that are garbled or silent (each also listed in the design notes):
 *   R1 FindZero's first argument is the end where the function is negative, the second the end
 *      where it is >= 0 (the call sites in Algorithm 3 pass them that way; the Require line is
 *      reversed).  It returns the negative-side end after the last iteration.
 *   R2 The Newton point is taken from the current negative end, t_neg^(i) - F/F', and clipped
 *      to the closed interval between the ORIGINAL negative end and the bisection point.  If the
 *      Newton point is not finite (F' = 0) the bisection point is used.
 *   R3 Stopping: exactly max_iter iterations (default 10) when tol = 0; with tol > 0 the loop
 *      also stops once the negative end moved by less than tol.
 *   R4 FindRange: the doubling starts at m = 0 (Algorithm 1); if F(t0 + 1) < 0 already, the
 *      returned positive end is t0 itself.  The number of doublings is capped (max_range).
 *   R5 Eq. (int) is read as log K = g(t_p) + log h + log sum_m c_m exp(g(t_m) - g(t_p)),
 *      the trapezoid rule of Sec. 2.4 (the printed form puts c_m in the exponent and h inside).
 *   R6 The derivative integrands reuse the forward range [t0, t1].
 *   R7 Inputs: v < 0 uses |v| (K is even in v) and flips the sign of d/dv; x = 0 gives
 *      log K = +inf, d/dv = 0 if v = 0 else +-inf, d/dx = -inf; x = +inf gives log K = -inf,
 *      d/dv = +-0, d/dx = -1; |v| = inf with finite x > 0 gives +inf, +-inf, -inf;
 *      x < 0 or a NaN gives NaN in all three outputs.
 *   R8 Second derivatives reuse the forward range too; x = +inf gives 0 for all three, every
 *      other edge input gives NaN.  d2/dv dx log K is odd in v (0 at v = 0), the other two even.
 */
#include <stdint.h>
#include <stdlib.h>
#include <tgmath.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef KV_REAL
#define KV_REAL double
#endif
#ifndef KV_SUFFIX
#define KV_SUFFIX d
#endif
#define KV_CAT2(a, b) a##_##b
#define KV_CAT(a, b) KV_CAT2(a, b)
#define KV_NAME(base) KV_CAT(base, KV_SUFFIX)

typedef KV_REAL real;

/* ---------------------------------------------------------------- Sec. 2.1: g and its t-derivatives */

typedef struct {
    real v, x;     /* order (already |v|) and argument */
    real G;        /* g(t_p), the offset of Eq. (int) */
    real log_eps;  /* log of the epsilon that defines the range (Sec. 2.1) */
} pair_t;

/* log cosh(a) written as |a| + log(1 + e^{-2|a|}) - log 2, which does not overflow. */
static real log_cosh(real a)
{
    a = fabs(a);
    return a + log1p(exp(-2 * a)) - log((real)2);
}

/* g(t) = log cosh(vt) - x cosh t */
static real g0(const pair_t* p, real t) { return log_cosh(p->v * t) - p->x * cosh(t); }

/* g'(t) = v tanh(vt) - x sinh t */
static real g1(const pair_t* p, real t) { return p->v * tanh(p->v * t) - p->x * sinh(t); }

/* g''(t) = v^2 sech^2(vt) - x cosh t */
static real g2(const pair_t* p, real t)
{
    real c = cosh(p->v * t);
    return p->v * p->v / (c * c) - p->x * cosh(t);
}

/* The two functions whose zeros Algorithm 3 looks for, with their t-derivatives:
 *   kind 0: F = g'  (the peak t_p),           F' = g''
 *   kind 1: F = h = g - g(t_p) - log eps,     F' = g'   (the ends t0, t1)                     */
static real F_of(const pair_t* p, int kind, real t)
{
    return kind == 0 ? g1(p, t) : g0(p, t) - p->G - p->log_eps;
}
static real dF_of(const pair_t* p, int kind, real t)
{
    return kind == 0 ? g2(p, t) : g1(p, t);
}

/* ---------------------------------------------------------------- Algorithm 1: FindRange */
/* Requires F(t0) >= 0.  Doubles m until F(t0 + 2^{m+1}) < 0 and returns
 * (t_pos, t_neg) = (t0 + 2^m, t0 + 2^{m+1}); reading R4 for the m = 0 exit. */
static void find_range(const pair_t* p, int kind, real t0, int max_range, real* t_pos, real* t_neg)
{
    int m = 0;
    while (m < max_range && F_of(p, kind, t0 + ldexp((real)1, m + 1)) >= 0)
        m++;
    real lo = t0 + ldexp((real)1, m);
    if (m == 0 && !(F_of(p, kind, lo) >= 0))
        lo = t0;
    *t_pos = lo;
    *t_neg = t0 + ldexp((real)1, m + 1);
}

/* ---------------------------------------------------------------- Algorithm 2: FindZero */
/* Bisection combined with a clipped Newton step (readings R1-R3). */
static real find_zero(const pair_t* p, int kind, real t_neg, real t_pos, int max_iter, real tol)
{
    real a = t_neg; /* current end with F < 0 */
    real b = t_pos; /* current end with F >= 0 */
    for (int i = 0; i < max_iter; i++) {
        real shrink = a + (b - a) / 2;
        real newton = a - F_of(p, kind, a) / dF_of(p, kind, a);
        if (!isfinite(newton))
            newton = shrink;
        real lo = fmin(t_neg, shrink), hi = fmax(t_neg, shrink);
        newton = fmin(fmax(newton, lo), hi);
        real a_prev = a;
        if (F_of(p, kind, shrink) < 0) {
            a = shrink;
        } else if (F_of(p, kind, newton) < 0) {
            a = newton;
            b = shrink;
        } else {
            b = newton;
        }
        if (tol > 0 && fabs(a - a_prev) < tol)
            break;
    }
    return a;
}

/* ---------------------------------------------------------------- reading R7 */
/* Returns 1 (and fills the outputs) if the pair is an edge case, 0 for a regular pair. */
static int edge_case(double v, double x, double* logk, double* dv, double* dx)
{
    if (isnan(v) || isnan(x) || x < 0) {
        *logk = *dv = *dx = NAN;
        return 1;
    }
    if (x == 0) {
        *logk = INFINITY;
        *dv = (v == 0) ? 0.0 : copysign(INFINITY, v);
        *dx = -INFINITY;
        return 1;
    }
    if (isinf(x)) {
        *logk = -INFINITY;
        *dv = copysign(0.0, v);
        *dx = -1.0;
        return 1;
    }
    if (isinf(v)) {
        *logk = INFINITY;
        *dv = copysign(INFINITY, v);
        *dx = -INFINITY;
        return 1;
    }
    return 0;
}

/* ---------------------------------------------------------------- Algorithm 3 + Eq. (int) */
/* One pair through the method.  brk (may be NULL) receives t0, t_p, t1, g(t_p). */
/* Second derivatives of an edge input (reading R8). */
static void edge_case2(double x, double* d2)
{
    const double z = isinf(x) && x > 0 ? 0.0 : NAN;
    d2[0] = d2[1] = d2[2] = z;
}

static void o1_pair(double v_in, double x_in, int bins, double log_eps, int max_iter, double tol,
                    int max_range, double* logk, double* dv, double* dx, double* brk, double* d2)
{
    if (edge_case(v_in, x_in, logk, dv, dx)) {
        if (brk) brk[0] = brk[1] = brk[2] = brk[3] = NAN;
        if (d2) edge_case2(x_in, d2);
        return;
    }
    pair_t p;
    real sign = v_in < 0 ? -1 : 1;
    p.v = fabs((real)v_in);
    p.x = (real)x_in;
    p.log_eps = (real)log_eps;
    p.G = 0;

    /* Sec. 2.2: the peak.  g''(0) = v^2 - x > 0 means g has a peak at t_p > 0. */
    real tp = 0;
    if (g2(&p, 0) > 0) {
        real ts, te;
        find_range(&p, 0, 0, max_range, &ts, &te);
        tp = find_zero(&p, 0, te, ts, max_iter, (real)tol);
    }
    p.G = g0(&p, tp);

    /* Sec. 2.3: t0 = 0 unless g(0) - g(t_p) <= log eps, then the zero of h in [0, t_p]. */
    real t0 = 0;
    if (g0(&p, 0) - p.G <= p.log_eps)
        t0 = find_zero(&p, 1, 0, tp, max_iter, (real)tol);

    /* t1: FindRange on h from t_p, then FindZero. */
    real ts, te;
    find_range(&p, 1, tp, max_range, &ts, &te);
    real t1 = find_zero(&p, 1, te, ts, max_iter, (real)tol);

    /* Sec. 2.4 Eq. (int), reading R5; Sec. 4.1 derivative integrands, reading R6. */
    real h = (t1 - t0) / bins;
    real s0 = 0, s1 = 0, s2 = 0, svv = 0, svx = 0, sxx = 0;
    for (int m = 0; m <= bins; m++) {
        real t = t0 + m * h;
        real c = (m == 0 || m == bins) ? (real)0.5 : (real)1;
        real w = c * exp(g0(&p, t) - p.G);
        s0 += w;
        s1 += w * t * tanh(p.v * t);
        s2 += w * cosh(t);
        if (d2) {
            svv += w * t * t;                          /* K_vv / (cosh(vt) e^{-x cosh t}) */
            svx += w * t * tanh(p.v * t) * cosh(t);    /* -K_vx / ... */
            sxx += w * cosh(t) * cosh(t);              /* K_xx / ... */
        }
    }
    *logk = (double)(p.G + log(h) + log(s0));
    *dv = (double)(sign * (s1 / s0));
    *dx = (double)(-(s2 / s0));
    if (d2) {
        /* reading R8: plain combinations of the same sums */
        const real ev = s1 / s0, ex = s2 / s0;
        d2[0] = (double)(svv / s0 - ev * ev);
        d2[1] = (double)(sign * (ex * ev - svx / s0));
        d2[2] = (double)(sxx / s0 - ex * ex);
    }
    if (brk) {
        brk[0] = (double)t0;
        brk[1] = (double)tp;
        brk[2] = (double)t1;
        brk[3] = (double)p.G;
    }
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Batched O1.  brk: NULL or 4 doubles per pair (t0, t_p, t1, g(t_p)); d2: NULL or 3 doubles per
 * pair (d2/dv2, d2/dv dx, d2/dx2 of log K). */
void KV_NAME(kv_oracle_o1)(const double* v, const double* x, int64_t n, int bins, double log_eps,
                           int max_iter, double tol, int max_range, double* logk, double* dv,
                           double* dx, double* brk, double* d2, int nthreads)
{
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++)
        o1_pair(v[i], x[i], bins, log_eps, max_iter, tol, max_range, logk + i, dv + i, dx + i,
                brk ? brk + 4 * i : NULL, d2 ? d2 + 3 * i : NULL);
}

/* Plain evaluation of g, g', g'' (for bracket invariant checks in the tests). */
void KV_NAME(kv_oracle_g)(double v, double x, const double* t, int64_t n, double* g, double* gp,
                          double* gpp)
{
    pair_t p = {fabs((real)v), (real)x, 0, 0};
    for (int64_t i = 0; i < n; i++) {
        g[i] = (double)g0(&p, (real)t[i]);
        gp[i] = (double)g1(&p, (real)t[i]);
        gpp[i] = (double)g2(&p, (real)t[i]);
    }
}

/* Algorithms 1 and 2 alone, for pinning them separately: kind 0 works on g', kind 1 on
 * h = g - G - log eps.  out[0..1] = FindRange(F, t_start), out[2] = FindZero(F, t_neg, t_pos). */
void KV_NAME(kv_oracle_alg12)(double v, double x, double G, double log_eps, int kind,
                              double t_start, double t_neg, double t_pos, int max_iter,
                              int max_range, double* out)
{
    pair_t p = {fabs((real)v), (real)x, (real)G, (real)log_eps};
    real a, b;
    find_range(&p, kind, (real)t_start, max_range, &a, &b);
    out[0] = (double)a;
    out[1] = (double)b;
    out[2] = (double)find_zero(&p, kind, (real)t_neg, (real)t_pos, max_iter, 0);
}

#ifdef KV_DENSE
/* ---------------------------------------------------------------- O2: dense adaptive quadrature */
/* Gauss-Legendre nodes on [-1, 1] as the roots of P_N, found by Newton's method on the three-term
 * recurrence (A&S 25.4.29 weights 2 / ((1 - z^2) P_N'(z)^2)).  Computed once, in long double. */
#define GL_N 20
static long double gl_z[GL_N], gl_w[GL_N];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    const long double pi = 3.14159265358979323846264338327950288L;
    for (int i = 0; i < GL_N; i++) {
        long double z = cosl(pi * (i + 0.75L) / (GL_N + 0.5L));
        long double dp = 1;
        for (int it = 0; it < 100; it++) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= GL_N; k++) {
                long double pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = GL_N * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-30L) break;
        }
        /* recompute P_N' at the converged root */
        long double p0 = 1, p1 = z;
        for (int k = 2; k <= GL_N; k++) {
            long double pk = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        dp = GL_N * (z * p1 - p0) / (z * z - 1);
        gl_z[i] = z;
        gl_w[i] = 2 / ((1 - z * z) * dp * dp);
    }
    gl_ready = 1;
}

typedef struct {
    long double v, x, gmax;
} dense_t;

static long double dense_g(const dense_t* d, long double t)
{
    long double a = fabsl(d->v * t);
    return a + log1pl(expl(-2 * a)) - logl(2.0L) - d->x * coshl(t);
}

/* integrals over [a, b] of e^{g - gmax} * {1, t tanh(vt), cosh t, t^2, t tanh(vt) cosh t,
 * cosh^2 t} by one GL panel */
#define NQ 6
static void gl_panel(const dense_t* d, long double a, long double b, long double out[NQ])
{
    long double c = (a + b) / 2, r = (b - a) / 2;
    for (int k = 0; k < NQ; k++) out[k] = 0;
    for (int i = 0; i < GL_N; i++) {
        long double t = c + r * gl_z[i];
        long double e = expl(dense_g(d, t) - d->gmax) * gl_w[i];
        long double th = tanhl(d->v * t), ch = coshl(t);
        out[0] += e;
        out[1] += e * t * th;
        out[2] += e * ch;
        out[3] += e * t * t;
        out[4] += e * t * th * ch;
        out[5] += e * ch * ch;
    }
    for (int k = 0; k < NQ; k++) out[k] *= r;
}

/* Adaptive bisection of [a, b]: a panel is accepted when its 20-point estimate and the sum of its
 * two halves agree to the panel's share of the tolerance, or to the rounding noise of the
 * integrand (about noise * |value|); at most 2^30 subdivisions deep. */
static void gl_adapt(const dense_t* d, long double a, long double b, const long double whole[NQ],
                     const long double tol[NQ], long double noise, int depth, long double acc[NQ])
{
    long double m = (a + b) / 2, l[NQ], r[NQ];
    gl_panel(d, a, m, l);
    gl_panel(d, m, b, r);
    int ok = 1;
    for (int k = 0; k < NQ; k++) {
        long double floor_k = noise * fabsl(l[k] + r[k]);
        if (fabsl(l[k] + r[k] - whole[k]) > fmaxl(tol[k], floor_k)) ok = 0;
    }
    if (ok || depth >= 30) {
        for (int k = 0; k < NQ; k++) acc[k] += l[k] + r[k];
        return;
    }
    long double half_tol[NQ];
    for (int k = 0; k < NQ; k++) half_tol[k] = tol[k] / 2;
    gl_adapt(d, a, m, l, half_tol, noise, depth + 1, acc);
    gl_adapt(d, m, b, r, half_tol, noise, depth + 1, acc);
}

static void o2_pair(double v_in, double x_in, double* logk, double* dv, double* dx, double* d2)
{
    if (edge_case(v_in, x_in, logk, dv, dx)) {
        if (d2) edge_case2(x_in, d2);
        return;
    }
    dense_t d;
    d.v = fabsl((long double)v_in);
    d.x = (long double)x_in;
    /* The peak: g is unimodal on [0, inf) and g' < 0 beyond asinh(v/x), where x sinh t > v. */
    long double lo = 0, hi = asinhl(d.v / d.x) + 1;
    const long double phi = 0.61803398874989484820458683436563812L;
    for (int it = 0; it < 300; it++) {
        long double m1 = hi - phi * (hi - lo), m2 = lo + phi * (hi - lo);
        if (dense_g(&d, m1) < dense_g(&d, m2)) lo = m1; else hi = m2;
    }
    long double tstar = (lo + hi) / 2;
    long double gstar = dense_g(&d, tstar);
    if (dense_g(&d, 0) > gstar) { tstar = 0; gstar = dense_g(&d, 0); }
    d.gmax = gstar;
    /* A range wide enough that the integrand outside it is below e^{-110} of its peak. */
    const long double cut = 110;
    long double step = 1.0L / 1024, b = tstar + step;
    while (dense_g(&d, b) - gstar > -cut) { step *= 2; b = tstar + step; }
    long double a = 0;
    if (dense_g(&d, 0) - gstar < -cut) {
        step = 1.0L / 1024;
        while (tstar - step > 0 && dense_g(&d, tstar - step) - gstar > -cut) step *= 2;
        a = tstar - step > 0 ? tstar - step : 0;
    }
    /* coarse total for the tolerance scale: 64 panels */
    long double total[NQ] = {0}, pan[NQ];
    for (int i = 0; i < 64; i++) {
        gl_panel(&d, a + (b - a) * i / 64, a + (b - a) * (i + 1) / 64, pan);
        for (int k = 0; k < NQ; k++) total[k] += pan[k];
    }
    long double tol[NQ], whole[NQ], acc[NQ] = {0};
    for (int k = 0; k < NQ; k++) tol[k] = 1e-18L * fabsl(total[k]);
    /* g is evaluated as the difference of terms up to |g(t_max)| + x cosh(b) in size */
    long double noise = 64 * LDBL_EPSILON * (1 + fabsl(gstar) + d.x * coshl(b) + d.v * b);
    gl_panel(&d, a, b, whole);
    gl_adapt(&d, a, b, whole, tol, noise, 0, acc);
    const long double sign = v_in < 0 ? -1 : 1;
    *logk = (double)(gstar + logl(acc[0]));
    *dv = (double)(sign * (acc[1] / acc[0]));
    *dx = (double)(-(acc[2] / acc[0]));
    if (d2) {
        const long double ev = acc[1] / acc[0], ex = acc[2] / acc[0];
        d2[0] = (double)(acc[3] / acc[0] - ev * ev);
        d2[1] = (double)(sign * (ex * ev - acc[4] / acc[0]));
        d2[2] = (double)(acc[5] / acc[0] - ex * ex);
    }
}

void kv_oracle_dense(const double* v, const double* x, int64_t n, double* logk, double* dv,
                     double* dx, double* d2, int nthreads)
{
    gl_init();
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; i++) o2_pair(v[i], x[i], logk + i, dv + i, dx + i, d2 ? d2 + 3 * i : NULL);
}
#endif
