"""The path in FP32 throughout (the plain bracket of Algorithms 1-3 in FP32, the 32-bit variant of
Sec. 4.2, with a float-float offset): against the oracle's method in long double at the same
bins and eps, on the hard band, the learned-bracket set, the whole target domain and edge
inputs; and as the learned path's fallback.

The FP32 range differs from the oracle's FP64 range by the FP32 searches and by a reference point
up to ln2/256 from the peak (the range is then wider by a fraction of a nat), so the comparison
is with the oracle's method error included: 2e-6 at 40 bins, the mixed path's bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from conftest import rel, rel_logk
from paper_2108_11560_gb300 import _native as N
from paper_2108_11560_gb300 import kv, learned
from paper_2108_11560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TOL = 2e-6


def _t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("workload", ["hard", "learned", "full"])
def test_f32_path_matches_oracle(workload):
    v, x = {"hard": lambda: W.hard_band(20000, seed=501), "learned": lambda: W.learned_bracket(20000, seed=502),
            "full": lambda: W.full_domain(20000, seed=503)}[workload]()
    v = np.concatenate([v, [0.0, 0.5, 1000.0, 1e-3, 7.5, -3.0]])
    x = np.concatenate([x, [1e-6, 1.0, 1e5, 1e-6, 7.5, 2.0]])
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    out = kv.kv_fwd_bwd_ex(_t(vf), _t(xf), bins=40, bracket="f32", status=True)
    ref = oracle.o1(v64, x64, bins=40, log_eps=-20.0, precision="long")
    st = out["status"].cpu().numpy()
    assert np.count_nonzero(st & N.KV_PAIR_FALLBACK) <= 2  # FP32 ranges are finite nearly always
    assert rel_logk(_np(out["logk"]), ref["logk"]).max() < TOL
    nz = v64 != 0
    assert np.all(_np(out["dv"])[~nz] == 0)
    assert rel(_np(out["dv"])[nz], ref["dv"][nz]).max() < TOL
    assert rel(_np(out["dx"]), ref["dx"]).max() < TOL
    truth = oracle.dense(v64[::20], x64[::20])
    assert rel_logk(_np(out["logk"])[::20], truth["logk"]).max() < TOL


def test_f32_path_second_derivatives():
    v, x = W.hard_band(8000, seed=504)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    out = kv.kv_fwd_bwd_ex(_t(vf), _t(xf), bins=40, bracket="f32", second=True)
    ref = oracle.o1(v64, x64, bins=40, log_eps=-20.0, precision="long", second=True)
    for k in ("d2v", "dvx", "d2x"):
        nz = ref[k] != 0
        assert rel(_np(out[k])[nz], ref[k][nz]).max() < TOL, k


def test_f32_path_edge_cases():
    v = np.array([1.0, 0.0, -2.0, 3.0, np.inf, 1.0, np.nan])
    x = np.array([0.0, 0.0, 0.0, np.inf, 1.0, -1.0, 1.0])
    out = kv.kv_fwd_bwd_ex(_t(v), _t(x), bins=32, bracket="f32", status=True)
    ref = kv.kv_fwd_bwd_ex(_t(v), _t(x), bins=32, bracket="plain")
    for k in ("logk", "dv", "dx"):
        a, b = _np(out[k]), _np(ref[k])
        assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)]), k
    assert np.all(out["status"].cpu().numpy() == N.KV_PAIR_EDGE)


def test_learned_fallback_through_the_f32_bracket():
    """A network with NaN outputs sends the pairs to the fallback, which now takes the FP32
    plain bracket: results within the mixed bound on the hard band and the extreme range.  (A
    few very narrow peaks survive: NaN predictions give a degenerate range at the peak that the
    check's Newton corrections can still carry into the window, a valid range.)"""
    bad = learned.Mlp.create(5)
    p = bad.params()
    p[-2:] = np.nan
    bad.set_params(p)
    v1, x1 = W.hard_band(10000, seed=505)
    v2, x2 = W.extreme_range(10000, seed=506)
    v = np.concatenate([v1, v2])
    x = np.concatenate([x1, x2])
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    out = kv.kv_fwd_bwd_ex(_t(vf), _t(xf), bins=64, bracket="mlp", mlp=bad, status=True)
    fb = (out["status"].cpu().numpy() & N.KV_PAIR_FALLBACK) != 0
    assert np.all(fb[:10000]) and fb.mean() > 0.99
    ref = oracle.o1(v64, x64, bins=64, log_eps=-20.0, precision="long")
    assert rel_logk(_np(out["logk"]), ref["logk"]).max() < TOL
    nz = v64 != 0
    assert rel(_np(out["dv"])[nz], ref["dv"][nz]).max() < TOL
    assert rel(_np(out["dx"]), ref["dx"]).max() < TOL
