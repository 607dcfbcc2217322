"""Second derivatives of log K (Sec. 4.1, the integrands f^(n,m) with n + m = 2) on the GPU: the
FP64 and mixed paths (plain and learned bracket, and the learned path's fallback) against the
oracle's same-bin second derivatives in long double, the Bessel equation on the GPU's own
outputs, the double-backward of log_besselk, the second backward epilogue, and edge inputs.

Tolerances (from the arithmetic of the shifted sums): FP64 1e-12 relative (the sums' rounding,
~130 terms x 2^-53, against variances that the shifts keep well conditioned; measured <= 5e-14);
mixed 2e-6 relative on the hard-band and learned-bracket workloads (FP32 weights and shifts to a
few 2^-24; measured <= 5e-7), and 2e-6 of the terms' scale (dv^2 + |d2v| etc.) on the whole
domain, where the learned range may differ from the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from conftest import rel
from paper_2108_11560_gb300 import _native as N
from paper_2108_11560_gb300 import kv, learned
from paper_2108_11560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
KEYS = ("d2v", "dvx", "d2x")
TOL_F64 = 1e-12
TOL_MIXED = 2e-6


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _scale(ref, k):
    return {"d2v": ref["dv"] ** 2 + np.abs(ref["d2v"]), "d2x": ref["dx"] ** 2 + np.abs(ref["d2x"]),
            "dvx": np.abs(ref["dv"] * ref["dx"]) + np.abs(ref["dvx"])}[k]


def _check(out, ref, v, tol, scaled=False):
    for k in KEYS:
        g = _np(out[k])
        if k == "dvx":
            assert np.all(g[v == 0] == 0)
        nz = ref[k] != 0
        e = np.abs(g[nz] - ref[k][nz]) / (_scale(ref, k)[nz] if scaled else np.abs(ref[k][nz]))
        assert e.max() < tol, (k, e.max())


@pytest.fixture(scope="module")
def net():
    return learned.default_network(DEV)


def test_fp64_second_derivatives_match_oracle():
    v1, x1 = W.full_domain(6000, seed=401)
    v2, x2 = W.hard_band(6000, seed=402)
    v = np.concatenate([v1, v2, [0.0, 0.5, 1000.0, 3.5, -2.0]])
    x = np.concatenate([x1, x2, [1e-6, 1.0, 1e5, 1e-3, 7.0]])
    out = kv.kv_fwd_bwd_ex(_t(v), _t(x), second=True)
    ref = oracle.o1(v, x, precision="long", second=True)
    _check(out, ref, v, TOL_F64)
    # the first derivatives of the same (shifted) sums
    assert rel(_np(out["dx"]), ref["dx"]).max() < 1e-13
    nz = v != 0
    assert rel(_np(out["dv"])[nz], ref["dv"][nz]).max() < 1e-13


@pytest.mark.parametrize("bracket", ["plain", "mlp"])
def test_mixed_second_derivatives_match_oracle(net, bracket):
    v1, x1 = W.hard_band(8000, seed=403)
    v2, x2 = W.learned_bracket(8000, seed=404)
    v = np.concatenate([v1, v2, [0.0, 0.5, 30.0, -4.0]])
    x = np.concatenate([x1, x2, [1e-2, 1.0, 40.0, 3.0]])
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=40, bracket=bracket,
                           mlp=net, second=True)
    ref = oracle.o1(v64, x64, bins=40, log_eps=-20.0, precision="long", second=True)
    _check(out, ref, v64, TOL_MIXED)
    # the whole target domain, on the terms' scale
    v, x = W.full_domain(8000, seed=405)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=40, bracket=bracket,
                           mlp=net, second=True)
    ref = oracle.o1(v64, x64, bins=40, log_eps=-20.0, precision="long", second=True)
    _check(out, ref, v64, TOL_MIXED, scaled=True)


def test_mixed_second_derivatives_through_the_fallback():
    """A network with NaN outputs sends every pair to the fallback kernel, which computes the
    second derivatives from the plain FP64 bracket."""
    bad = learned.Mlp.create(5)
    p = bad.params()
    p[-2:] = np.nan
    bad.set_params(p)
    v, x = W.hard_band(3000, seed=406)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=40, bracket="mlp",
                           mlp=bad, second=True, status=True)
    assert np.all(out["status"].cpu().numpy() & N.KV_PAIR_FALLBACK)
    ref = oracle.o1(v64, x64, bins=40, log_eps=-20.0, precision="long", second=True)
    _check(out, ref, v64, TOL_MIXED)


def test_bessel_equation_on_gpu_outputs():
    """x^2 K'' + x K' - (x^2 + v^2) K = 0: L'' = 1 + v^2/x^2 - L'/x - L'^2 from the FP64 path's
    own first and second x-derivatives."""
    v, x = W.full_domain(4000, seed=407)
    out = kv.kv_fwd_bwd_ex(_t(v), _t(x), second=True)
    d1, d2 = _np(out["dx"]), _np(out["d2x"])
    rhs = 1 + (v / x) ** 2 - d1 / x - d1 * d1
    scale = 1 + (v / x) ** 2 + np.abs(d1) / x + d1 * d1
    assert np.max(np.abs(d2 - rhs) / scale) < 1e-13


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_double_backward_hessian_vector_product(net, dtype):
    """grad of (a . dL/dv + b . dL/dx) with respect to (v, x) through log_besselk's differentiable
    backward equals the second derivatives applied to (a, b), element by element."""
    v, x = W.hard_band(5000, seed=408)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    if dtype == torch.float64:
        v64, x64 = v, x
        vt, xt, kw, tol = _t(v), _t(x), {}, TOL_F64
        ref = oracle.o1(v, x, precision="long", second=True)
    else:
        vt, xt = _t(vf, dtype), _t(xf, dtype)
        kw, tol = {"bins": 40, "bracket": "mlp", "mlp": net}, TOL_MIXED
        ref = oracle.o1(v64, x64, bins=40, log_eps=-20.0, precision="long", second=True)
    vt.requires_grad_(True)
    xt.requires_grad_(True)
    rng = np.random.default_rng(409)
    a, b = rng.uniform(-1, 1, v.size), rng.uniform(-1, 1, v.size)
    lk = kv.log_besselk(vt, xt, **kw)
    gv, gx = torch.autograd.grad(lk.sum(), (vt, xt), create_graph=True)
    hv, hx = torch.autograd.grad((gv * _t(a, dtype)).sum() + (gx * _t(b, dtype)).sum(), (vt, xt))
    want_v = a * ref["d2v"] + b * ref["dvx"]
    want_x = a * ref["dvx"] + b * ref["d2x"]
    sv = np.abs(a) * _scale(ref, "d2v") + np.abs(b) * _scale(ref, "dvx")
    sx = np.abs(a) * _scale(ref, "dvx") + np.abs(b) * _scale(ref, "d2x")
    assert np.max(np.abs(_np(hv) - want_v) / sv) < tol
    assert np.max(np.abs(_np(hx) - want_x) / sx) < tol


def test_second_backward_epilogue():
    rng = np.random.default_rng(410)
    n = 10007
    arrs = [_t(rng.normal(size=n)) for _ in range(8)]
    go, ggv, ggx, dv, dx, d2v, dvx, d2x = arrs
    ov, ox, ogo = kv.kv_grad2(go, ggv, ggx, dv, dx, d2v, dvx, d2x)
    G = [_np(t) for t in arrs]
    assert np.allclose(_np(ov), G[0] * (G[1] * G[5] + G[2] * G[6]), rtol=1e-15, atol=1e-15)
    assert np.allclose(_np(ox), G[0] * (G[1] * G[6] + G[2] * G[7]), rtol=1e-15, atol=1e-15)
    assert np.allclose(_np(ogo), G[1] * G[3] + G[2] * G[4], rtol=1e-15, atol=1e-15)
    ov, ox, ogo = kv.kv_grad2(go, None, ggx, dv, dx, d2v, dvx, d2x)
    assert np.allclose(_np(ov), G[0] * G[2] * G[6], rtol=1e-15, atol=1e-15)


def test_second_derivatives_edge_cases(net):
    v = np.array([1.0, 2.0, np.nan, 1.0, np.inf, 0.0])
    x = np.array([np.inf, 0.0, 1.0, -1.0, 1.0, 2.0])
    for dtype, kw in ((torch.float64, {}), (torch.float32, {}), (torch.float32, {"bracket": "mlp", "mlp": net})):
        out = kv.kv_fwd_bwd_ex(_t(v, dtype), _t(x, dtype), second=True, **kw)
        for k in KEYS:
            g = _np(out[k])
            assert g[0] == 0 and np.all(np.isnan(g[1:5])), (dtype, kw, k, g)
        assert _np(out["dvx"])[5] == 0  # v = 0
