"""The seeded input generators (paper_2108_11560_gb300/workloads.py) draw what their recipes say:
ranges, proportions, the hard band's structure, the special orders of the extreme range, the
paper's grids, and the same values for the same seed (runs without a GPU)."""
import numpy as np

from paper_2108_11560_gb300 import workloads as W


def test_same_seed_same_inputs():
    a = W.hard_band(10_000, seed=11)
    b = W.hard_band(10_000, seed=11)
    c = W.hard_band(10_000, seed=12)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


def test_uniform_small():
    v, x = W.uniform_small()
    assert v.size == x.size == 4096
    assert v.min() >= 0 and v.max() <= 10 and x.min() >= 1e-2 and x.max() <= 1e2


def test_hard_band_structure():
    n = 200_000
    v, x = W.hard_band(n, seed=1)
    assert v.size == x.size == n and v.min() >= 0 and v.max() <= 50
    assert x.min() >= 1e-3 and x.max() <= 1e3 * (1 + 1e-12)
    band = np.abs(x - v) <= 0.1 * v + 1e-3
    # a quarter of the pairs are drawn in the band; the bulk lands there only rarely
    assert 0.25 <= band.mean() < 0.27
    # shuffled: the band is spread over the whole array
    q = band.reshape(10, -1).mean(axis=1)
    assert q.min() > 0.2 and q.max() < 0.32


def test_gh_likelihood_ranges():
    lam, x, alpha, delta, z = W.gh_likelihood(50_000, seed=2)
    assert lam.dtype == np.float32 and x.dtype == np.float32
    assert lam.min() >= -5 and lam.max() <= 5 and alpha.min() >= 0.5 and delta.max() <= 3
    ref = delta.astype(np.float64) * alpha * np.sqrt(1 + z.astype(np.float64) ** 2)
    assert np.allclose(x, ref, rtol=1e-6)


def test_extreme_range_special_orders():
    v, x = W.extreme_range(400_000, seed=5)
    zero = v == 0
    half = (v > 0) & (np.abs(v - np.floor(v) - 0.5) < 1e-12) & (v < 1000)
    assert 0.009 < zero.mean() < 0.011
    assert 0.009 < half.mean() < 0.012
    rest = v[~zero & ~half]
    assert rest.min() >= 1e-3 and rest.max() <= 1e3
    assert x.min() >= 1e-6 and x.max() <= 1e5


def test_paper_grids():
    v, x = W.paper_scaling(100_000, seed=8)
    assert v.min() >= 0 and v.max() <= 99 and x.min() >= 0.1 and x.max() <= 100
    gv, gx = W.paper_accuracy_grid()
    assert gv.size == gx.size == 81 * 125
    assert gv.min() == 0 and np.isclose(gv.max(), 99)
    assert np.isclose(gx.min(), 0.1) and np.isclose(gx.max(), 10 ** 2.1)


def test_to_f32_gives_both_sides_the_cast_values():
    v = np.array([0.1, 1 / 3, 2.0 ** -30])
    (vf, v64), = W.to_f32(v)
    assert vf.dtype == np.float32 and v64.dtype == np.float64
    assert np.array_equal(v64, vf.astype(np.float64))
