"""Pins of the learned-bracket oracle (oracle/mlp.py) to facts outside itself (no GPU)."""
import os

import numpy as np

from oracle import mlp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_params(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, mlp.NPARAMS)


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.uniform(0, 200, n)
    x = 10 ** rng.uniform(-4, 4, n)
    tp = rng.uniform(0, 10, n) * (rng.uniform(0, 1, n) > 0.3)
    t0 = np.maximum(tp - rng.uniform(0, 3, n), 0)
    t1 = tp + rng.uniform(0.01, 5, n)
    return v, x, t0, tp, t1


def test_gradient_matches_central_differences():
    """Every one of the 4482 partial derivatives against a central difference of the loss."""
    p = _rand_params(1)
    v, x, t0, tp, t1 = _batch(24, 2)
    _, g = mlp.loss_grad(p, v, x, t0, tp, t1)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp.loss_grad(p + e, v, x, t0, tp, t1)
        lm, _ = mlp.loss_grad(p - e, v, x, t0, tp, t1)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    assert np.count_nonzero(g) > 1000  # the ReLUs leave most units active


def test_zero_network_outputs_bias_only():
    p = np.zeros(mlp.NPARAMS)
    d = mlp.unpack(p)
    d["b3"][:] = [0.25, -0.5]
    p = mlp.pack(d)
    y = mlp.forward(p, [1.0, 50.0], [0.1, 10.0])["y"]
    assert np.array_equal(y, [[0.25, -0.5], [0.25, -0.5]])
    v, x, t0, tp, t1 = _batch(5, 3)
    _, g = mlp.loss_grad(p, v, x, t0, tp, t1)
    G = mlp.unpack(g)
    assert np.all(G["W1"] == 0) and np.all(G["W2"] == 0) and np.all(G["W3"] == 0)
    T = mlp.targets(t0, tp, t1)
    assert np.allclose(G["b3"], (np.array([0.25, -0.5]) - T).mean(0), rtol=1e-14)


def test_targets_invert_predict():
    """A network whose outputs equal the targets predicts the target bracket back."""
    v, x, t0, tp, t1 = _batch(50, 4)
    T = mlp.targets(t0, tp, t1)
    d = mlp.unpack(np.zeros(mlp.NPARAMS))
    out = []
    for i in range(50):
        d["b3"][:] = T[i]
        out.append(mlp.predict(mlp.pack(d), v[i:i + 1], x[i:i + 1], tp[i:i + 1]))
    p0 = np.array([o[0][0] for o in out])
    p1 = np.array([o[1][0] for o in out])
    assert np.allclose(p0, t0, atol=1e-12) and np.allclose(p1, t1, atol=1e-12)


def test_adam_first_step_closed_form():
    """From zero moments the first Adam step is -lr * g / (|g| + eps) (bias correction exact)."""
    p = _rand_params(5)
    g = np.random.default_rng(6).normal(0, 1e-3, p.size)
    p1, m, s = mlp.adam(p, np.zeros_like(p), np.zeros_like(p), g, 1, 1e-3, 0.9, 0.999, 1e-8)
    assert np.allclose(p1 - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(s, 0.001 * g * g)


def test_splitmix64_reference_outputs():
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    golden = 0x9E3779B97F4A7C15
    got = [mlp.mix64((1234567 + k * golden) & mlp.MASK64) for k in range(5)]
    assert got == want


def test_batch_indices_in_range_and_spread():
    idx = mlp.batch_indices(7, 3, 4096, 1000)
    assert idx.min() >= 0 and idx.max() < 1000
    assert len(np.unique(idx)) > 950
    # consecutive steps draw different samples; twenty small batches cover nearly the whole set
    a, b = mlp.batch_indices(7, 0, 64, 1000), mlp.batch_indices(7, 1, 64, 1000)
    assert len(np.intersect1d(a, b)) < 20
    seen = np.unique(np.concatenate([mlp.batch_indices(7, j, 256, 1000) for j in range(20)]))
    assert len(seen) > 990


def test_training_reduces_loss():
    """A few hundred Adam steps on a smooth synthetic bracket lower the loss."""
    rng = np.random.default_rng(8)
    n = 4096
    v = rng.uniform(0, 200, n)
    x = 10 ** rng.uniform(-4, 4, n)
    tp = np.arcsinh(np.maximum(v, 1e-3) / x) * (v * v > x)
    t0 = np.maximum(tp - 1.0 / np.sqrt(1 + x), 0)
    t1 = tp + 3.0 / np.sqrt(1 + x)
    p0 = _rand_params(9, 0.2)
    p, losses = mlp.train(p0, v, x, t0, t1, steps=300, batch=256, lr=3e-3, beta1=0.9,
                          beta2=0.999, eps=1e-8, seed=10)
    assert losses[-20:].mean() < 0.2 * losses[:5].mean()


def test_peak_is_the_zero_of_g_prime():
    """The reference point of the learned bracket: the zero of g' (brentq), 0 when v^2 <= x."""
    import scipy.optimize

    import oracle
    rng = np.random.default_rng(11)
    v = np.concatenate([rng.uniform(0, 1000, 150), [1.0, 2.0, 0.0]])
    x = np.concatenate([10 ** rng.uniform(-6, 5, 150), [1.0, 3.99, 1.0]])
    t = mlp.peak(v, x)
    for i in range(v.size):
        if v[i] ** 2 <= x[i]:
            assert t[i] == 0
            continue
        g = lambda s: oracle.g_eval(v[i], x[i], [s], precision="long")[1][0]
        root = scipy.optimize.brentq(g, 1e-300, 64.0, xtol=1e-15)
        assert abs(t[i] - root) <= 1e-9 * max(1.0, root)
