"""Per-(v, x) time maps (Sec. 3.2) on a small grid: every path finishes every point, the times
are positive and finite, and the learned and FP32 paths stay within a small factor of their own
median everywhere (the flat map the paper reports for the integration method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2108_11560_gb300 import timemap

pytestmark = pytest.mark.gpu


def test_grid_is_the_papers_thinned():
    vs, xs = timemap.grid(9, 9)
    assert vs[0] == 0 and np.isclose(vs[-1], 99.0) and np.isclose(xs[0], 0.1) and np.isclose(xs[-1], 10 ** 2.1)


def test_small_time_map():
    maps = timemap.time_map(("f32", "learned", "fp64"), pairs=1 << 16, nv=3, nx=3, reps=2)
    for name, (vs, xs, t) in maps.items():
        assert t.shape == (3, 3) and np.all(np.isfinite(t)) and np.all(t > 0), name
        text = timemap.format_map(vs, xs, t)
        assert text.count("\n") == 3
    for name in ("f32", "learned"):
        t = maps[name][2]
        assert t.max() < 8 * np.median(t), (name, t)
