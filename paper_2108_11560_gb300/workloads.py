"""Seeded synthetic (v, x) inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the method: it only draws inputs with numpy's PCG64
(``numpy.random.default_rng(seed)``), in float64 on the host.  Each generator is named for the
workload it stands for; sizes are arguments so tests can draw small slices of the same recipe.
The paper uses no public dataset (its accuracy reference was Mathematica; Sec. 3), so every
input here is synthetic.
"""
from __future__ import annotations

import numpy as np


def uniform_small(n: int = 4096, seed: int = 0):
    """v ~ U[0, 10], x log-uniform in [1e-2, 1e2] (the 4096-pair FP64 plain-method case)."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(0.0, 10.0, n)
    x = 10.0 ** rng.uniform(-2.0, 2.0, n)
    return v, x


def hard_band(n: int = 16_777_216, seed: int = 1, band_frac: float = 0.25):
    """75 %: v ~ U[0, 50], x log-uniform in [1e-3, 1e3]; 25 %: the band |v - x| < 0.1 v,
    x = v (1 + 0.1 U[-1, 1]) clamped to x >= 1e-3; shuffled (the 16M-pair mixed-vs-FP64 case)."""
    rng = np.random.default_rng(seed)
    nb = int(round(n * band_frac))
    na = n - nb
    v = np.empty(n)
    x = np.empty(n)
    v[:na] = rng.uniform(0.0, 50.0, na)
    x[:na] = 10.0 ** rng.uniform(-3.0, 3.0, na)
    vb = rng.uniform(0.0, 50.0, nb)
    v[na:] = vb
    x[na:] = np.maximum(vb * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, nb)), 1e-3)
    perm = rng.permutation(n)
    return v[perm], x[perm]


def gh_likelihood(n: int = 8_388_608, seed: int = 2):
    """Generalized-hyperbolic-style samples: order lam ~ U[-5, 5], z ~ N(0, 1), alpha ~ U[0.5, 5],
    delta ~ U[0.1, 3], argument x = delta * alpha * sqrt(1 + z^2).  Returns float32 arrays
    (lam, x, alpha, delta, z)."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-5.0, 5.0, n)
    z = rng.standard_normal(n)
    alpha = rng.uniform(0.5, 5.0, n)
    delta = rng.uniform(0.1, 3.0, n)
    x = delta * alpha * np.sqrt(1.0 + z * z)
    f = np.float32
    return lam.astype(f), x.astype(f), alpha.astype(f), delta.astype(f), z.astype(f)


def learned_bracket(n: int, seed: int = 3):
    """v ~ U[0, 200], x log-uniform in [1e-4, 1e4] (training set of the learned bracket; the
    64M-pair evaluation set uses a fresh seed)."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(0.0, 200.0, n)
    x = 10.0 ** rng.uniform(-4.0, 4.0, n)
    return v, x


def learned_bracket_mixed(n: int, seed: int = 3):
    """The learned-bracket inputs with half of the orders log-uniform in [1e-3, 200] instead of
    uniform, so that small orders (v < 1) are represented; x log-uniform in [1e-4, 1e4]."""
    v, x = learned_bracket(n, seed)
    rng = np.random.default_rng(seed + 1000)
    k = n // 2
    v[:k] = 10.0 ** rng.uniform(-3.0, np.log10(200.0), k)
    return v, x


def extreme_range(n: int = 134_217_728, seed: int = 5):
    """v log-uniform in [1e-3, 1e3] except 1 % v = 0 exactly and 1 % v = k + 1/2, k ~ U{0..999};
    x log-uniform in [1e-6, 1e5] (the 128M-pair extreme-range case)."""
    rng = np.random.default_rng(seed)
    v = 10.0 ** rng.uniform(-3.0, 3.0, n)
    sel = rng.uniform(0.0, 1.0, n)
    v[sel < 0.01] = 0.0
    half = (sel >= 0.01) & (sel < 0.02)
    v[half] = rng.integers(0, 1000, int(half.sum())) + 0.5
    x = 10.0 ** rng.uniform(-6.0, 5.0, n)
    return v, x


def extreme_training(n: int, seed: int = 4):
    """Training inputs for a network covering the extreme range: half of the orders log-uniform
    in [1e-3, 1e3], half uniform in [0, 1000]; x log-uniform in [1e-6, 1e5]."""
    rng = np.random.default_rng(seed)
    k = n // 2
    v = np.concatenate([10.0 ** rng.uniform(-3.0, 3.0, k), rng.uniform(0.0, 1000.0, n - k)])
    x = 10.0 ** rng.uniform(-6.0, 5.0, n)
    return v, x


def full_domain(n: int, seed: int = 7):
    """v ~ U[0, 1000], x log-uniform in [1e-6, 1e5] (the accuracy targets' whole domain)."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(0.0, 1000.0, n)
    x = 10.0 ** rng.uniform(-6.0, 5.0, n)
    return v, x


def paper_scaling(n: int, seed: int = 8):
    """The paper's vectorised-timing inputs (Sec. 3.4): v = 10^{2 r1} - 1 in [0, 99] and
    x = 10^{3 r2 - 1} in [0.1, 100] with independent r1, r2 ~ U(0, 1)."""
    rng = np.random.default_rng(seed)
    v = 10.0 ** (2.0 * rng.uniform(0.0, 1.0, n)) - 1.0
    x = 10.0 ** (3.0 * rng.uniform(0.0, 1.0, n) - 1.0)
    return v, x


def paper_accuracy_grid(step: int = 1):
    """The accuracy-map grid of Sec. 3 over the range it states, v in [0, 99] and
    x in [10^-1, 10^2.1]: v = 10^{i/40} - 1, i = 0..80 and x = 10^{(i - 40)/40}, i = 0..124 (125
    points a fortieth of a decade apart; the exponent i/40 alone would start the axis at 1), every
    ``step``-th point on each axis.  Returns flattened (v, x)."""
    v = 10.0 ** (np.arange(0, 81, step) / 40.0) - 1.0
    x = 10.0 ** ((np.arange(0, 125, step) - 40) / 40.0)
    vv, xx = np.meshgrid(v, x, indexing="ij")
    return vv.ravel(), xx.ravel()


def to_f32(*arrays):
    """Cast to float32 and return float64 copies of the cast values, so that both sides of a
    comparison see exactly the same inputs."""
    out = []
    for a in arrays:
        f = np.asarray(a, dtype=np.float32)
        out.append((f, f.astype(np.float64)))
    return out
