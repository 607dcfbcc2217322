"""Pins of the CPU oracle to facts outside itself (no GPU).

The oracle (O1: the fixed-bin method of Sec. 2 / Algorithm 3; O2: dense adaptive quadrature)
is checked against closed forms, Bessel identities, an independent high-precision quadrature
(mpmath), a brute-force long-double trapezoid and the bracket definitions of Sec. 2.1-2.3.
Each check is chosen so that a plausible slip in the oracle (a dropped c_0 = 1/2, a sign, a
wrong factor in g', g'', a transposed bracket end, a missing log h) fails at least one of them.
"""
import math

import mpmath
import numpy as np
import pytest
import scipy.optimize
import scipy.special

import oracle
from conftest import rel, rel_logk
from paper_2108_11560_gb300 import workloads as W

mpmath.mp.dps = 40

# tolerances: the FP64 method's own rounding (|g| up to 1e5 enters each bin) versus the same
# steps in long double, and the long double results against exact values.
TOL_LONG_LOGK = 1e-14
TOL_LONG_DERIV = 1e-13
TOL_F64_LOGK = 1e-13
TOL_F64_DERIV = 2e-11


def _all_oracles(v, x, bins=128):
    return {
        "o1_double": oracle.o1(v, x, bins=bins, precision="double"),
        "o1_long": oracle.o1(v, x, bins=bins, precision="long"),
        "dense": oracle.dense(v, x),
    }


def _tols(name):
    if name == "o1_double":
        return TOL_F64_LOGK, TOL_F64_DERIV
    return TOL_LONG_LOGK, TOL_LONG_DERIV


# ------------------------------------------------------------------ closed forms

def _log_k_half(k, x):
    """log K_{k+1/2}(x) = log[ sqrt(pi/2x) e^{-x} sum_{j=0}^{k} (k+j)! / (j! (k-j)! (2x)^j) ]."""
    x = mpmath.mpf(x)
    s = mpmath.fsum(mpmath.factorial(k + j) / (mpmath.factorial(j) * mpmath.factorial(k - j) * (2 * x) ** j)
                    for j in range(k + 1))
    return mpmath.log(mpmath.sqrt(mpmath.pi / (2 * x)) * mpmath.exp(-x) * s)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 5, 8])
def test_half_integer_closed_form(k):
    """K_{k+1/2} is elementary; d/dx log K follows from K' = -(K_{v-1} + K_{v+1}) / 2 with
    K_{-1/2} = K_{1/2}.  Covers both branches of Sec. 2.2 (v^2 <= x and v^2 > x)."""
    xs = np.array([1e-3, 0.05, 0.3, 1.0, 7.5, 40.0, 300.0, 1e4])
    v = np.full_like(xs, k + 0.5)
    ref_l = np.array([float(_log_k_half(k, xx)) for xx in xs])
    ref_dx = []
    for xx in xs:
        lo = _log_k_half(abs(k - 1), xx) if k >= 1 else _log_k_half(0, xx)  # K_{v-1}: v-1 = k-1/2
        hi = _log_k_half(k + 1, xx)
        mid = _log_k_half(k, xx)
        ref_dx.append(float(-(mpmath.exp(lo - mid) + mpmath.exp(hi - mid)) / 2))
    ref_dx = np.array(ref_dx)
    for name, out in _all_oracles(v, xs).items():
        tl, td = _tols(name)
        assert rel_logk(out["logk"], ref_l).max() < tl, name
        assert rel(out["dx"], ref_dx).max() < td, name


def test_dv_at_half_closed_form():
    """d/dv log K_v(x) at v = 1/2 equals e^{2x} E_1(2x) (from dK_v/dv at v = 1/2, DLMF 10.38.7)."""
    xs = np.array([1e-4, 1e-2, 0.3, 1.0, 4.0, 25.0, 200.0])
    ref = np.array([float(mpmath.exp(2 * mpmath.mpf(xx)) * mpmath.e1(2 * mpmath.mpf(xx))) for xx in xs])
    for name, out in _all_oracles(np.full_like(xs, 0.5), xs).items():
        _, td = _tols(name)
        assert rel(out["dv"], ref).max() < td, name
        # and the order -1/2: d/dv is odd in v
        neg = oracle.o1(np.full_like(xs, -0.5), xs, precision="long")
    assert rel(-neg["dv"], ref).max() < TOL_LONG_DERIV


def test_mpmath_besselk_small_orders():
    """mpmath's besselk at orders v <= 20, where it agrees with its own quadrature."""
    rng = np.random.default_rng(100)
    v = rng.uniform(0, 20, 40)
    x = 10 ** rng.uniform(-4, 3, 40)
    ref = np.array([float(mpmath.log(mpmath.besselk(a, b))) for a, b in zip(v, x)])
    for name, out in _all_oracles(v, x).items():
        tl, _ = _tols(name)
        assert rel_logk(out["logk"], ref).max() < tl, name


def _mp_quad_logk(v, x):
    """log of the integral of Eq. (1)-(2) by mpmath tanh-sinh quadrature, with breakpoints
    around the maximum of log f found on a plain grid (independent of Algorithms 1-3)."""
    v = mpmath.mpf(v)
    x = mpmath.mpf(x)
    lg = lambda t: mpmath.log(mpmath.cosh(v * t)) - x * mpmath.cosh(t)
    # beyond asinh(v/x) g decreases; beyond acosh(1 + 130/x) it has fallen by more than 120
    top = max(float(mpmath.asinh(v / x)), float(mpmath.acosh(1 + 130 / x))) + 1
    grid = np.linspace(0, top, 4001)
    vals = [float(lg(mpmath.mpf(t))) for t in grid]
    i = int(np.argmax(vals))
    gmax = vals[i]
    keep = [t for t, g in zip(grid, vals) if g > gmax - 120]
    a, b = keep[0], keep[-1]
    a = max(0.0, a - (grid[1] - grid[0]))
    b = b + (grid[1] - grid[0])
    pts = [mpmath.mpf(p) for p in np.linspace(a, b, 17)]
    I = mpmath.quad(lambda t: mpmath.exp(lg(t) - gmax), pts)
    return float(gmax + mpmath.log(I))


@pytest.mark.slow
def test_mpmath_quadrature_full_domain():
    """Independent quadrature of Eq. (1)-(2) at 30 digits on a sample of v in [0, 1000],
    x in [1e-6, 1e5] (mpmath's besselk itself is unreliable at some large orders)."""
    mpmath.mp.dps = 30
    try:
        v, x = W.full_domain(24, seed=101)
        v = np.concatenate([v, [1000.0, 1000.0, 0.0, 0.0, 459.71597989318457]])
        x = np.concatenate([x, [1e-6, 1e5, 1e-6, 1e5, 301.2442190495824]])
        ref = np.array([_mp_quad_logk(a, b) for a, b in zip(v, x)])
    finally:
        mpmath.mp.dps = 40
    for name, out in _all_oracles(v, x).items():
        tl, _ = _tols(name)
        assert rel_logk(out["logk"], ref).max() < max(tl, 1e-14), name


def test_mpmath_numerical_dv():
    """d/dv log K by mpmath's numerical differentiation of log besselk (small orders)."""
    pts = [(0.3, 0.01), (1.7, 1.0), (4.2, 30.0), (12.5, 3.0), (7.0, 1e3)]
    v = np.array([p[0] for p in pts])
    x = np.array([p[1] for p in pts])
    ref = np.array([float(mpmath.diff(lambda s: mpmath.log(mpmath.besselk(s, b)), a)) for a, b in pts])
    for name, out in _all_oracles(v, x).items():
        _, td = _tols(name)
        assert rel(out["dv"], ref).max() < td, name


# ------------------------------------------------------------------ identities

def test_symmetry_in_v():
    """K_{-v} = K_v: log K and d/dx are even in v, d/dv is odd and exactly 0 at v = 0."""
    v, x = W.full_domain(300, seed=102)
    for prec in ("double", "long"):
        a = oracle.o1(v, x, precision=prec)
        b = oracle.o1(-v, x, precision=prec)
        assert np.array_equal(a["logk"], b["logk"])
        assert np.array_equal(a["dx"], b["dx"])
        assert np.array_equal(a["dv"], -b["dv"])
        z = oracle.o1(np.zeros(20), 10 ** np.linspace(-6, 5, 20), precision=prec)
        assert np.all(z["dv"] == 0.0)
    d = oracle.dense(-v[:50], x[:50])
    assert rel_logk(d["logk"], a["logk"][:50]).max() < TOL_LONG_LOGK


def test_recurrence():
    """K_{v+1} = K_{v-1} + (2v/x) K_v, i.e. e^{L(v+1)-L(v)} = e^{L(v-1)-L(v)} + 2v/x."""
    rng = np.random.default_rng(103)
    v = rng.uniform(1.0, 300.0, 200)
    x = 10 ** rng.uniform(-5, 4, 200)
    for prec, tol in (("long", 1e-13), ("double", 1e-11)):
        lm = oracle.o1(v - 1, x, precision=prec)["logk"]
        l0 = oracle.o1(v, x, precision=prec)["logk"]
        lp = oracle.o1(v + 1, x, precision=prec)["logk"]
        lhs = np.exp(lp - l0)
        rhs = np.exp(lm - l0) + 2 * v / x
        # log K is returned in FP64: its rounding enters e^{L(v+1) - L(v)} as 2^-53 |L|
        rounding = 2.0 ** -52 * (np.abs(lm) + np.abs(l0) + np.abs(lp))
        assert (rel(lhs, rhs) / (tol + rounding)).max() < 1, prec


def test_dx_identity():
    """d/dx log K_v = -(e^{L(v-1)-L(v)} + e^{L(v+1)-L(v)}) / 2 = -v/x - e^{L(v-1)-L(v)} (Eq. deriv,
    read with d log K / dx on the left)."""
    v, x = W.full_domain(300, seed=104)
    v = v + 1.0
    for prec, tol in (("long", 1e-13), ("double", 1e-11)):
        lm = oracle.o1(v - 1, x, precision=prec)["logk"]
        r0 = oracle.o1(v, x, precision=prec)
        lp = oracle.o1(v + 1, x, precision=prec)["logk"]
        l0 = r0["logk"]
        ref = -(np.exp(lm - l0) + np.exp(lp - l0)) / 2
        rounding = 2.0 ** -52 * (np.abs(lm) + np.abs(l0) + np.abs(lp))
        assert (rel(r0["dx"], ref) / (tol + rounding)).max() < 1, prec
        assert (rel(r0["dx"], -v / x - np.exp(lm - l0)) / (tol + rounding)).max() < 1, prec


def test_scipy_kve_sanity():
    """scipy's FP64 kve (library routine) at moderate orders, to 1e-12."""
    rng = np.random.default_rng(105)
    v = rng.uniform(0, 30, 200)
    x = 10 ** rng.uniform(-2, 3, 200)
    ref = np.log(scipy.special.kve(v, x)) - x
    out = oracle.o1(v, x, precision="long")
    assert rel_logk(out["logk"], ref).max() < 1e-12


# ------------------------------------------------------------------ brute force

def test_bruteforce_trapezoid_long_double():
    """Trapezoid with 200k bins on a wide fixed range in numpy long double (tiny grid)."""
    pts = [(0.0, 1e-3), (0.5, 2.0), (3.0, 0.1), (20.0, 25.0), (80.0, 1.0), (250.0, 400.0)]
    ld = np.longdouble
    for v, x in pts:
        top = math.asinh(max(v, 1.0) / x) + 6.0
        t = np.linspace(ld(0), ld(top), 200_001, dtype=ld)
        a = np.abs(ld(v) * t)
        g = a + np.log1p(np.exp(-2 * a)) - np.log(ld(2)) - ld(x) * np.cosh(t)
        gm = g.max()
        w = np.exp(g - gm)
        w[0] *= ld(0.5)
        w[-1] *= ld(0.5)
        hstep = t[1] - t[0]
        s0 = w.sum()
        ref_l = float(gm + np.log(hstep * s0))
        ref_dv = float((w * t * np.tanh(ld(v) * t)).sum() / s0)
        ref_dx = float(-(w * np.cosh(t)).sum() / s0)
        out = oracle.o1([v], [x], precision="long")
        assert rel_logk(out["logk"], ref_l)[0] < 1e-14, (v, x)
        assert rel(out["dx"], ref_dx)[0] < 1e-13, (v, x)
        if v > 0:
            assert rel(out["dv"], ref_dv)[0] < 1e-13, (v, x)


@pytest.mark.parametrize("bins, log_eps", [(1, -3.0), (2, -3.0), (5, -8.0), (128, oracle.LOG_EPS_F64)])
def test_fixed_bins_on_returned_bracket_match_library_trapezoid(bins, log_eps):
    """Eq. (int) given the bracket: on the [t0, t1] that the oracle returns, log K and the two
    derivative ratios equal scipy's composite trapezoid over bins + 1 equally spaced points
    (bins = 1 is the textbook two-point rule).  With a coarse eps the range end matters, so a
    wrong bin width or a dropped end weight shows even where the integrand is tiny."""
    import scipy.integrate
    v, x = W.full_domain(40, seed=111)
    v = np.concatenate([v, [0.0, 0.5, 30.0]])
    x = np.concatenate([x, [2.0, 0.1, 40.0]])
    out = oracle.o1(v, x, bins=bins, log_eps=log_eps, precision="long", bracket=True)
    ld = np.longdouble
    for i in range(v.size):
        t0, t1 = ld(out["t0"][i]), ld(out["t1"][i])
        if not t1 > t0:
            continue
        t = t0 + (t1 - t0) * np.arange(bins + 1, dtype=ld) / ld(bins)
        a = np.abs(ld(v[i]) * t)
        g = a + np.log1p(np.exp(-2 * a)) - np.log(ld(2)) - ld(x[i]) * np.cosh(t)
        gm = g.max()
        w = np.exp(g - gm)
        s0 = scipy.integrate.trapezoid(w, t)
        ref_l = float(gm + np.log(s0))
        ref_dv = float(scipy.integrate.trapezoid(w * t * np.tanh(ld(v[i]) * t), t) / s0)
        ref_dx = float(-scipy.integrate.trapezoid(w * np.cosh(t), t) / s0)
        # t0, t1 come back rounded to FP64: the points above are those rounded ends
        assert rel_logk(out["logk"][i:i + 1], ref_l)[0] < 1e-12, (v[i], x[i])
        assert rel(out["dx"][i:i + 1], ref_dx)[0] < 1e-11, (v[i], x[i])
        if v[i] > 0:
            assert rel(out["dv"][i:i + 1], ref_dv)[0] < 1e-11, (v[i], x[i])


def test_o1_against_dense_full_domain():
    """The method at 128 bins against the dense quadrature on the whole target domain."""
    v, x = W.full_domain(2000, seed=106)
    d = oracle.dense(v, x)
    lo = oracle.o1(v, x, precision="long")
    assert rel_logk(lo["logk"], d["logk"]).max() < TOL_LONG_LOGK
    assert rel(lo["dv"], d["dv"]).max() < TOL_LONG_DERIV
    assert rel(lo["dx"], d["dx"]).max() < TOL_LONG_DERIV
    db = oracle.o1(v, x, precision="double")
    assert rel_logk(db["logk"], d["logk"]).max() < TOL_F64_LOGK
    assert rel(db["dv"], d["dv"]).max() < TOL_F64_DERIV
    assert rel(db["dx"], d["dx"]).max() < TOL_F64_DERIV


def test_bins_convergence():
    """Sec. 2.4: a fixed number of bins over the eps-range; the error falls fast with n and
    stays at rounding level from 64 bins on (the FP64 target needs n >= 48 here)."""
    v, x = W.full_domain(1000, seed=107)
    d = oracle.dense(v, x)
    errs = {n: rel_logk(oracle.o1(v, x, bins=n, precision="long")["logk"], d["logk"]).max()
            for n in (16, 32, 64, 128)}
    assert errs[16] > errs[32] > 1e-15
    assert errs[64] < 1e-14 and errs[128] < 1e-14


# ------------------------------------------------------------------ brackets (Sec. 2.1-2.3, Alg. 1-2)

def test_bracket_invariants():
    """t0 <= t_p <= t1; t_p = 0 iff v^2 <= x; h(t0) <= 0 unless t0 = 0; h(t1) < 0; the peak
    lies within the final FindZero step of the true zero of g' (scipy brentq)."""
    v, x = W.full_domain(400, seed=108)
    v = np.concatenate([v, [0.0, 1.0, 1e-3, 10.0]])
    x = np.concatenate([x, [1.0, 1.0, 1e-6, 100.0]])
    out = oracle.o1(v, x, precision="long", bracket=True)
    le = oracle.LOG_EPS_F64
    for i in range(v.size):
        t0, tp, t1, G = out["t0"][i], out["tp"][i], out["t1"][i], out["G"][i]
        assert 0 <= t0 <= tp <= t1
        g, gp, gpp = oracle.g_eval(v[i], x[i], [0.0, t0, tp, t1], precision="long")
        assert G == g[2]
        if np.longdouble(v[i]) ** 2 <= np.longdouble(x[i]):  # g''(0) = v^2 - x <= 0
            assert tp == 0
        else:
            # the negative-side end of g' (up to the FP64 rounding of t_p on the way out)
            assert tp > 0 and gp[2] <= 4 * np.spacing(tp) * abs(gpp[2])
            f = lambda t: oracle.g_eval(v[i], x[i], [t], precision="long")[1][0]
            root = scipy.optimize.brentq(f, 1e-300, 64.0, xtol=1e-15, maxiter=500) if f(64.0) < 0 else None
            if root is not None:
                assert abs(tp - root) <= 2.0 ** -10 * 32
        # the values come back rounded to FP64: allow that rounding of G and of t
        tt = np.array([0.0, t0, tp, t1])
        slack = 4 * 2.0 ** -52 * (abs(G) + np.abs(g)) + 4 * np.spacing(tt) * np.abs(gp)
        if t0 > 0:
            assert g[1] - G - le <= slack[1]
        assert g[3] - G - le < slack[3]
        assert g[0] - G - le <= slack[0] or t0 == 0


def test_findrange_and_findzero_alone():
    """Algorithm 1 returns a positive and a negative end 2^m apart; Algorithm 2 returns a point
    where F < 0 within 2^-10 of the initial width of the zero found by brentq."""
    rng = np.random.default_rng(109)
    for _ in range(200):
        v = float(rng.uniform(0.5, 1000))
        x = float(10 ** rng.uniform(-6, math.log10(v * v) - 1e-3))
        pos, neg, z = oracle.alg12(v, x, 0, 0.0, 0.0, 0.0, precision="long")
        gp = lambda t: oracle.g_eval(v, x, [t], precision="long")[1][0]
        assert gp(pos) >= 0 and gp(neg) < 0
        assert neg - pos == (2.0 if pos == 0 else pos)  # (2^m, 2^{m+1}) or (0, 2)
        _, _, tp = oracle.alg12(v, x, 0, 0.0, neg, pos, precision="long")
        # g'(0) = 0 exactly: start the reference search just above 0, where g' > 0
        root = scipy.optimize.brentq(gp, pos if pos > 0 else 1e-300, neg, xtol=1e-15)
        gpp = oracle.g_eval(v, x, [tp], precision="long")[2][0]
        assert gp(tp) <= 4 * np.spacing(tp) * abs(gpp) and tp >= root - 4 * np.spacing(root)
        assert tp - root <= (neg - pos) * 2.0 ** -10


def test_findzero_keeps_the_zero_bracketed():
    """Algorithm 2 on h = g - G - log eps from a negative end just above 0, where h' is tiny
    and a full Newton step lands far beyond the bracket: the result stays in the initial
    bracket, on its negative side, within 2^-10 of its width of the zero there (brentq)."""
    le = oracle.LOG_EPS_F64
    for v, x in [(1000.0, 1.0), (50.0, 0.01), (300.0, 20.0), (5.0, 1e-4)]:
        o = oracle.o1([v], [x], precision="long", bracket=True)
        tp, G = o["tp"][0], o["G"][0]
        for t_neg in (1e-8, 1e-5):
            h = lambda t: oracle.g_eval(v, x, [t], precision="long")[0][0] - G - le
            assert h(t_neg) < 0 < h(tp)
            _, _, z = oracle.alg12(v, x, 1, 0.0, t_neg, tp, G=G, log_eps=le, precision="long")
            r = scipy.optimize.brentq(h, t_neg, tp, xtol=1e-15)
            assert t_neg <= z <= tp, (v, x, t_neg, z)
            # z comes back rounded to FP64: allow that rounding on the negative side
            slope = abs(oracle.g_eval(v, x, [z], precision="long")[1][0])
            assert h(z) <= 4 * np.spacing(z) * slope, (v, x, t_neg, z)
            assert r - z <= (tp - t_neg) * 2.0 ** -10, (v, x, t_neg, z, r)


def test_stopping_rule_reading():
    """Reading of the stopping rule: fixed 10 iterations (tol = 0) and a tolerance stop at
    1e-8 give the same results to the FP64 target (Sec. 1: a coarse range is enough)."""
    v, x = W.full_domain(500, seed=110)
    a = oracle.o1(v, x, precision="long", tol=0.0)
    b = oracle.o1(v, x, precision="long", tol=1e-8)
    assert rel_logk(a["logk"], b["logk"]).max() < 1e-13


def test_edge_cases():
    """x = 0, x = inf, v = +-inf, x < 0 and NaN inputs."""
    v = np.array([1.0, 0.0, -2.0, 3.0, -3.0, np.inf, -np.inf, 1.0, np.nan, 1.0, 0.0])
    x = np.array([0.0, 0.0, 0.0, np.inf, np.inf, 1.0, 1.0, -1.0, 1.0, np.nan, np.inf])
    for out in (oracle.o1(v, x), oracle.o1(v, x, precision="long"), oracle.dense(v, x)):
        lk, dv, dx = out["logk"], out["dv"], out["dx"]
        assert lk[0] == np.inf and dv[0] == np.inf and dx[0] == -np.inf
        assert lk[1] == np.inf and dv[1] == 0 and dx[1] == -np.inf
        assert lk[2] == np.inf and dv[2] == -np.inf
        assert lk[3] == -np.inf and dv[3] == 0 and dx[3] == -1 and not np.signbit(dv[3])
        assert np.signbit(dv[4])
        assert lk[5] == np.inf and dv[5] == np.inf and dx[5] == -np.inf
        assert lk[6] == np.inf and dv[6] == -np.inf
        for i in (7, 8, 9):
            assert np.isnan(lk[i]) and np.isnan(dv[i]) and np.isnan(dx[i])


def test_paper_error_metric():
    """The paper's accuracy scale log10(|Delta|/eps + 1) (Sec. 3) of O1 against the dense
    quadrature on its own accuracy grid: below 1 everywhere for log K (Sec. 3.1) and d/dx
    (Sec. 4.1)."""
    v, x = W.paper_accuracy_grid(step=4)
    d = oracle.dense(v, x)
    o = oracle.o1(v, x, precision="double")
    eps = 2.0 ** -52
    err = lambda a, b: np.log10(np.abs(a - b) / (eps * np.maximum(np.abs(b), 1e-300)) + 1)
    # relative deviation in units of eps (log K itself, as the paper compares values of K)
    assert np.median(err(o["logk"], d["logk"])) < 1
    assert np.median(err(o["dx"], d["dx"])) < 1


# ------------------------------------------------------------------ second derivatives (Sec. 4.1, n + m = 2)

@pytest.mark.parametrize("k", [0, 1, 3, 6])
def test_second_dx_half_integer_closed_form(k):
    """d2/dx2 log K_{k+1/2}(x) by mpmath differentiation of the elementary closed form
    (for k = 0 it is 1/(2x^2))."""
    xs = np.array([1e-3, 0.05, 0.7, 3.0, 40.0, 300.0, 1e4])
    ref = np.array([float(mpmath.diff(lambda t: _log_k_half(k, t), mpmath.mpf(xx), 2)) for xx in xs])
    if k == 0:
        assert np.allclose(ref, 1 / (2 * xs ** 2), rtol=4e-16, atol=0)
    for name, out in (("o1_long", oracle.o1(np.full_like(xs, k + 0.5), xs, precision="long", second=True)),
                      ("dense", oracle.dense(np.full_like(xs, k + 0.5), xs, second=True))):
        # the plain combination E[cosh^2] - E[cosh]^2 cancels to ~1/(2x^2): the sums of ~130
        # terms in long double (2^-64) leave about 130 2^-64 E[cosh]^2 absolute in it
        tol = 1e-12 + 1e3 * 2.0 ** -64 * out["dx"] ** 2 / ref
        assert np.all(rel(out["d2x"], ref) < tol), (name, rel(out["d2x"], ref))


def test_second_dx_bessel_equation():
    """x^2 K'' + x K' - (x^2 + v^2) K = 0 in log form: L'' = 1 + v^2/x^2 - L'/x - L'^2, with L'
    the (pinned) first derivative, on the whole target domain."""
    v, x = W.full_domain(300, seed=120)
    o = oracle.o1(v, x, precision="long", second=True)
    d1 = o["dx"]
    rhs = 1 + (v / x) ** 2 - d1 / x - d1 * d1
    scale = 1 + (v / x) ** 2 + np.abs(d1) / x + d1 * d1
    assert np.max(np.abs(o["d2x"] - rhs) / scale) < 1e-14


def test_second_dvx_recurrence_identity():
    """d/dx log K_v = -v/x - R with R = K_{v-1}/K_v (Eq. deriv, corrected); its v-derivative:
    d2/dv dx log K_v = -1/x - R (d/dv log K_{v-1} - d/dv log K_v)."""
    rng = np.random.default_rng(121)
    v = rng.uniform(0.0, 300.0, 300)
    x = 10 ** rng.uniform(-4, 4, 300)
    a = oracle.o1(v, x, precision="long", second=True)
    b = oracle.o1(v - 1, x, precision="long")
    R = np.exp(b["logk"] - a["logk"])
    rhs = -1 / x - R * (b["dv"] - a["dv"])
    scale = 1 / x + R * (np.abs(b["dv"]) + np.abs(a["dv"]))
    assert np.max(np.abs(a["dvx"] - rhs) / scale) < 1e-12


def _mp_second_v(v, x):
    """d2/dv2 log K by mpmath quadrature of K, K_v and K_vv (30 digits)."""
    v = mpmath.mpf(v)
    x = mpmath.mpf(x)
    f = lambda t: mpmath.exp(-x * mpmath.cosh(t))
    top = max(float(mpmath.asinh(v / x)), float(mpmath.acosh(1 + 80 / x))) + 2
    pts = [mpmath.mpf(p) for p in np.linspace(0, top, 129)]  # panels narrower than the peak
    K = mpmath.quad(lambda t: mpmath.cosh(v * t) * f(t), pts)
    Kv = mpmath.quad(lambda t: t * mpmath.sinh(v * t) * f(t), pts)
    Kvv = mpmath.quad(lambda t: t * t * mpmath.cosh(v * t) * f(t), pts)
    return float(Kvv / K - (Kv / K) ** 2)


def test_second_dv_mpmath_quadrature():
    """d2/dv2 log K against an independent mpmath quadrature at small orders."""
    mpmath.mp.dps = 30
    try:
        pts = [(0.0, 0.3), (0.5, 1.0), (2.5, 0.05), (7.0, 20.0), (15.0, 3.0), (30.0, 100.0)]
        ref = np.array([_mp_second_v(a, b) for a, b in pts])
    finally:
        mpmath.mp.dps = 40
    v = np.array([p[0] for p in pts])
    x = np.array([p[1] for p in pts])
    for out in (oracle.o1(v, x, precision="long", second=True), oracle.dense(v, x, second=True)):
        assert rel(out["d2v"], ref).max() < 1e-12


def test_second_derivatives_symmetry_and_signs():
    """d2v and d2x are even in v, dvx is odd and 0 at v = 0; d2x > 0 (log K is convex in x)
    and d2v > 0 (K_v(x) is log-convex in v)."""
    v, x = W.full_domain(300, seed=122)
    a = oracle.o1(v, x, precision="long", second=True)
    b = oracle.o1(-v, x, precision="long", second=True)
    assert np.array_equal(a["d2v"], b["d2v"]) and np.array_equal(a["d2x"], b["d2x"])
    assert np.array_equal(a["dvx"], -b["dvx"])
    z = oracle.o1(np.zeros(10), 10 ** np.linspace(-6, 5, 10), precision="long", second=True)
    assert np.all(z["dvx"] == 0)
    assert np.all(a["d2x"] > 0) and np.all(a["d2v"] > 0)


def test_second_derivatives_o1_against_dense():
    """The method's second derivatives at 128 bins against the dense quadrature; the plain
    combinations cancel to about 1/(2 x^2) at large x, so the bound scales with the terms."""
    v, x = W.full_domain(1000, seed=123)
    d = oracle.dense(v, x, second=True)
    lo = oracle.o1(v, x, precision="long", second=True)
    e1 = lo["dv"] ** 2 + np.abs(d["d2v"])
    assert np.max(np.abs(lo["d2v"] - d["d2v"]) / e1) < 1e-12
    e2 = lo["dx"] ** 2 + np.abs(d["d2x"])
    assert np.max(np.abs(lo["d2x"] - d["d2x"]) / e2) < 1e-12
    e3 = np.abs(lo["dx"] * lo["dv"]) + np.abs(d["dvx"])
    assert np.max(np.abs(lo["dvx"] - d["dvx"]) / e3) < 1e-12


def test_second_derivatives_edge_cases():
    v = np.array([1.0, 2.0, np.nan, 1.0, np.inf])
    x = np.array([np.inf, 0.0, 1.0, -1.0, 1.0])
    for out in (oracle.o1(v, x, second=True), oracle.o1(v, x, precision="long", second=True),
                oracle.dense(v, x, second=True)):
        for k in ("d2v", "dvx", "d2x"):
            assert out[k][0] == 0
            assert np.all(np.isnan(out[k][1:]))
