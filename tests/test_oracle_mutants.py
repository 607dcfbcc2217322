"""Planted mistakes: each mutant is a copy of the oracle's C source (or of its MLP module) with
one plausible slip (a dropped endpoint weight, a sign, a wrong end returned by FindZero, a missing
factor in a derivative integrand, a transposed weight in the backward pass, ...).  Every mutant
must fail at least one of the pins in test_oracle_pins.py / test_oracle_mlp.py, which shows the
pins constrain every part of the oracle.  Runs on the CPU."""
import json
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "kv_oracle.c")

# (name, text in kv_oracle.c, replacement): each text occurs exactly once
MUTANTS = [
    ("endpoint weight 1/2 dropped", "(m == 0 || m == bins) ? (real)0.5 : (real)1", "(real)1"),
    ("log h dropped", "*logk = (double)(p.G + log(h) + log(s0));", "*logk = (double)(p.G + log(s0));"),
    ("log 2 dropped in log cosh", "return a + log1p(exp(-2 * a)) - log((real)2);", "return a + log1p(exp(-2 * a));"),
    ("sign of x sinh in g'", "return p->v * tanh(p->v * t) - p->x * sinh(t); }", "return p->v * tanh(p->v * t) + p->x * sinh(t); }"),
    ("v instead of v^2 in g''", "return p->v * p->v / (c * c) - p->x * cosh(t);", "return p->v / (c * c) - p->x * cosh(t);"),
    ("FindZero returns the positive end", "    return a;\n}\n\n/* ---------------------------------------------------------------- reading R7 */",
     "    return b;\n}\n\n/* ---------------------------------------------------------------- reading R7 */"),
    ("Newton step with the wrong sign", "real newton = a - F_of(p, kind, a) / dF_of(p, kind, a);",
     "real newton = a + F_of(p, kind, a) / dF_of(p, kind, a);"),
    ("FindRange negative end 2^m", "*t_neg = t0 + ldexp((real)1, m + 1);", "*t_neg = t0 + ldexp((real)1, m);"),
    ("t0 test inverted", "if (g0(&p, 0) - p.G <= p.log_eps)", "if (g0(&p, 0) - p.G > p.log_eps)"),
    ("t missing in the d/dv integrand", "s1 += w * t * tanh(p.v * t);", "s1 += w * tanh(p.v * t);"),
    ("sinh for cosh in the d/dx integrand", "s2 += w * cosh(t);", "s2 += w * sinh(t);"),
    ("d/dv sign not flipped for v < 0", "real sign = v_in < 0 ? -1 : 1;", "real sign = 1;"),
    ("bin width over n + 1", "real h = (t1 - t0) / bins;", "real h = (t1 - t0) / (bins + 1);"),
    ("peak bracket ends swapped", "tp = find_zero(&p, 0, te, ts, max_iter, (real)tol);",
     "tp = find_zero(&p, 0, ts, te, max_iter, (real)tol);"),
    ("FindRange keeps t0 + 1 when m = 0", "if (m == 0 && !(F_of(p, kind, lo) >= 0))",
     "if (0 && !(F_of(p, kind, lo) >= 0))"),
    ("bisection keeps the wrong half", "            a = shrink;\n        } else if", "            b = shrink;\n        } else if"),
    ("Newton step not clipped", "newton = fmin(fmax(newton, lo), hi);", "(void)lo; (void)hi;"),
    ("five FindZero iterations", "for (int i = 0; i < max_iter; i++) {", "for (int i = 0; i < max_iter - 5; i++) {"),
    ("offset G missing from h", "g0(p, t) - p->G - p->log_eps;", "g0(p, t) - p->log_eps;"),
    ("x = inf gives d/dx = 0", "*dx = -1.0;", "*dx = 0.0;"),
    ("x = 0 loses the sign of v", "*dv = (v == 0) ? 0.0 : copysign(INFINITY, v);", "*dv = (v == 0) ? 0.0 : INFINITY;"),
    ("Gauss-Legendre weights halved", "gl_w[i] = 2 / ((1 - z * z) * dp * dp);", "gl_w[i] = 1 / ((1 - z * z) * dp * dp);"),
    ("Gauss-Legendre panel not scaled", "for (int k = 0; k < NQ; k++) out[k] *= r;", ""),
    ("dense d/dv integrand without t", "out[1] += e * t * th;", "out[1] += e * th;"),
    ("dense range starts at the peak", "a = tstar - step > 0 ? tstar - step : 0;", "a = tstar;"),
    ("K_vv integrand with t for t^2", "svv += w * t * t;", "svv += w * t;"),
    ("K_vx integrand without cosh t", "svx += w * t * tanh(p.v * t) * cosh(t);", "svx += w * t * tanh(p.v * t);"),
    ("K_xx integrand with cosh t once", "sxx += w * cosh(t) * cosh(t);", "sxx += w * cosh(t);"),
    ("d2v without the square of d/dv", "d2[0] = (double)(svv / s0 - ev * ev);", "d2[0] = (double)(svv / s0);"),
    ("dvx not odd in v", "d2[1] = (double)(sign * (ex * ev - svx / s0));", "d2[1] = (double)((ex * ev - svx / s0));"),
    ("dvx with the product's sign flipped", "d2[1] = (double)(sign * (ex * ev - svx / s0));", "d2[1] = (double)(sign * (-ex * ev - svx / s0));"),
    ("dense K_xx integrand with cosh t once", "out[5] += e * ch * ch;", "out[5] += e * ch;"),
    ("dense d2x plus the square", "d2[2] = (double)(acc[5] / acc[0] - ex * ex);", "d2[2] = (double)(acc[5] / acc[0] + ex * ex);"),
    ("second derivatives 0 for every edge input", "const double z = isinf(x) && x > 0 ? 0.0 : NAN;", "const double z = 0.0;"),
]

# the pins run against each mutant (the ones that take well under a second each)
PINS = [
    lambda: pins.test_half_integer_closed_form(0),
    lambda: pins.test_half_integer_closed_form(3),
    pins.test_dv_at_half_closed_form,
    pins.test_mpmath_besselk_small_orders,
    pins.test_symmetry_in_v,
    pins.test_recurrence,
    pins.test_dx_identity,
    pins.test_bruteforce_trapezoid_long_double,
    lambda: pins.test_fixed_bins_on_returned_bracket_match_library_trapezoid(1, -3.0),
    lambda: pins.test_fixed_bins_on_returned_bracket_match_library_trapezoid(5, -8.0),
    pins.test_o1_against_dense_full_domain,
    pins.test_bracket_invariants,
    pins.test_findrange_and_findzero_alone,
    pins.test_findzero_keeps_the_zero_bracketed,
    pins.test_edge_cases,
    lambda: pins.test_second_dx_half_integer_closed_form(1),
    pins.test_second_dx_bessel_equation,
    pins.test_second_dvx_recurrence_identity,
    pins.test_second_dv_mpmath_quadrature,
    pins.test_second_derivatives_symmetry_and_signs,
    pins.test_second_derivatives_o1_against_dense,
    pins.test_second_derivatives_edge_cases,
]


def _caught_here(mutant_libs):
    with oracle.swap_libraries(mutant_libs):
        for pin in PINS:
            try:
                pin()
            except Exception:  # an assertion, or the mutant producing NaN/inf where it should not
                return True
    return False


def _caught(mutant_libs, timeout=60):
    """Runs the pins against the mutant in a child process: a mutant that makes the oracle run
    without end (an adaptive quadrature that never accepts a panel) counts as caught once the
    child runs past the time limit, and the child is then killed."""
    code = ("import sys, json; sys.path[:0] = json.loads(sys.argv[1]); "
            "import test_oracle_mutants as t; "
            "sys.exit(3 if t._caught_here(json.loads(sys.argv[2])) else 0)")
    paths = [os.path.dirname(os.path.abspath(__file__)), os.path.dirname(os.path.dirname(os.path.abspath(__file__)))]
    try:
        r = subprocess.run([sys.executable, "-c", code, json.dumps(paths), json.dumps(mutant_libs)],
                           capture_output=True, text=True, timeout=timeout)
    except subprocess.TimeoutExpired:
        return True
    assert r.returncode in (0, 3), r.stderr[-2000:]
    return r.returncode == 3


def test_pins_pass_on_the_oracle_itself():
    for pin in PINS:
        pin()


@pytest.mark.parametrize("name, old, new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_every_planted_mistake_is_caught(name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    d = tempfile.mkdtemp(prefix="kv_oracle_mutant_")
    try:
        path = os.path.join(d, "kv_oracle.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        libs = oracle.compile_variant_source(path, d)
        assert _caught(libs), f"no pin catches: {name}"
    finally:
        shutil.rmtree(d, ignore_errors=True)
    # the real oracle is back in place
    pins.test_half_integer_closed_form(0)


# ------------------------------------------------------------------ the learned-bracket oracle

MLP_SRC = os.path.join(os.path.dirname(oracle.__file__), "mlp.py")

MLP_MUTANTS = [
    ("backward through W2 transposed", 'dz1 = (dz2 @ P["W2"])', 'dz1 = (dz2 @ P["W2"].T)'),
    ("layer-2 ReLU mask from layer 1", '* (F["z2"] > 0)', '* (F["z1"] > 0)'),
    ("b1 gradient from layer 2", 'g["b1"] = dz1.sum(0)', 'g["b1"] = dz2.sum(0)'),
    ("W1 gradient with the features swapped", 'g["W1"] = dz1.T @ F["f"]', 'g["W1"] = dz1.T @ F["f"][:, ::-1]'),
    ("loss not halved", "loss = 0.5 * np.sum(r * r) / B", "loss = np.sum(r * r) / B"),
    ("Adam without bias correction", "mh = m / (1 - beta1 ** step)", "mh = m"),
    ("Adam second moment of |g|", "s = beta2 * s + (1 - beta2) * g * g", "s = beta2 * s + (1 - beta2) * np.abs(g)"),
    ("Adam steps uphill", "return p - lr * mh", "return p + lr * mh"),
    ("target L1 measured from t0", "L1 = np.log(np.maximum(np.asarray(t1) - np.asarray(tp), 0.0) + DELTA)",
     "L1 = np.log(np.maximum(np.asarray(t1) - np.asarray(t0), 0.0) + DELTA)"),
    ("predict scales L1 like L0", "L1 = y[:, 1] * OUT_SCALE[2] + OUT_SCALE[3]", "L1 = y[:, 1] * OUT_SCALE[0] + OUT_SCALE[1]"),
    ("predict keeps DELTA", "t1 = t_ref + np.maximum(np.exp(L1) - DELTA, 0.0)", "t1 = t_ref + np.exp(L1)"),
    ("peak Newton step with the wrong sign", "t = np.clip(t - step, 0.0, t)", "t = np.clip(t + step, 0.0, t)"),
    ("SplitMix64 last shift 33", "return z ^ (z >> 31)", "return z ^ (z >> 33)"),
    ("batch indices ignore the step", "mix64((seed + step * batch + k) & MASK64)", "mix64((seed + k) & MASK64)"),
]


def _mlp_pins():
    import test_oracle_mlp as t
    return t, [getattr(t, name) for name in dir(t) if name.startswith("test_")]


@pytest.mark.parametrize("name, old, new", MLP_MUTANTS, ids=[m[0] for m in MLP_MUTANTS])
def test_every_planted_mlp_mistake_is_caught(name, old, new):
    import types
    src = open(MLP_SRC).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle.mlp_mutant")
    exec(compile(src.replace(old, new), MLP_SRC, "exec"), mod.__dict__)
    t, tests = _mlp_pins()
    saved = t.mlp
    t.mlp = mod
    caught = False
    try:
        for pin in tests:
            try:
                pin()
            except Exception:
                caught = True
                break
    finally:
        t.mlp = saved
    assert caught, f"no pin catches: {name}"


def test_mlp_pins_pass_on_the_oracle_itself():
    _, tests = _mlp_pins()
    for pin in tests:
        pin()
