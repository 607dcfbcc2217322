"""Host logic of the time maps (paper_2108_11560_gb300/timemap.py), without a GPU: the grid is the
paper's evaluation grid of Sec. 3 (v = 10^(i/40) - 1 for i = 0..80, x = 10^(i/40) for
i = -40..84) thinned with both ends kept, and the table has one row per order."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2108_11560_gb300 import timemap  # noqa: E402


def test_grid_keeps_the_ends_of_the_papers_domain():
    vs, xs = timemap.grid(9, 9)
    assert vs.size == 9 and xs.size == 9
    assert vs[0] == 0.0 and np.isclose(vs[-1], 99.0)
    assert np.isclose(xs[0], 0.1) and np.isclose(xs[-1], 10 ** 2.1)
    assert np.all(np.diff(vs) > 0) and np.all(np.diff(xs) > 0)
    # the full grid: 81 orders and 125 arguments
    vf, xf = timemap.grid(81, 125)
    assert vf.size == 81 and xf.size == 125
    assert np.allclose(vf, 10 ** (np.arange(81) / 40) - 1)
    assert np.allclose(xf, 10 ** (np.arange(-40, 85) / 40))


def test_format_map_has_a_row_per_order():
    vs, xs = timemap.grid(3, 4)
    t = np.arange(12, dtype=float).reshape(3, 4) / 7
    text = timemap.format_map(vs, xs, t)
    lines = text.splitlines()
    assert len(lines) == 1 + vs.size
    assert all(len(l.split()) == 1 + xs.size for l in lines[1:])
