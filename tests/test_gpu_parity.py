"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

FP64 path: within 1e-13 relative of the oracle's fixed-bin method computed in long double
(log K relative to max(1, |log K|); d/dv and d/dx plain relative; d/dv = 0 exactly at v = 0).
Mixed path: within 2e-6 of the same method in long double at the mixed path's eps, and of the
dense-quadrature truth.  Sizes span several warps and a ragged tail; edge cases included.
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
TOL_F64 = 1e-13
TOL_MIXED = 2e-6
MIXED_LOG_EPS = -20.0


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _deriv_ok(gpu, ref, v, tol):
    """plain relative error; where v = 0 both must be exactly 0."""
    z = v == 0
    assert np.all(gpu[z] == 0.0)
    return rel(gpu[~z], ref[~z]).max() if (~z).any() else 0.0


# ------------------------------------------------------------------ FP64 path

def test_fp64_small_uniform_logk():
    """4096 pairs, v ~ U[0, 10], x log-uniform [1e-2, 1e2], 128 bins, log K only."""
    v, x = W.uniform_small(4096, seed=0)
    ref = oracle.o1(v, x, bins=128, precision="long")
    lk = _np(kv.kv_log(_t(v), _t(x), bins=128))
    assert rel_logk(lk, ref["logk"]).max() < TOL_F64


@pytest.mark.parametrize("bins", [48, 128])
def test_fp64_fwd_bwd_full_domain(bins):
    """v in [0, 1000], x in [1e-6, 1e5] plus the hard band, all three outputs."""
    v1, x1 = W.full_domain(6000, seed=201)
    v2, x2 = W.hard_band(3000, seed=202)
    v = np.concatenate([v1, v2, [0.0, 0.5, 1000.0, 1000.0, 0.0]])
    x = np.concatenate([x1, x2, [1e-6, 1.0, 1e-6, 1e5, 1e5]])
    ref = oracle.o1(v, x, bins=bins, precision="long")
    lk, dv, dx = (_np(t) for t in kv.kv_fwd_bwd(_t(v), _t(x), bins=bins))
    assert rel_logk(lk, ref["logk"]).max() < TOL_F64
    assert _deriv_ok(dv, ref["dv"], v, TOL_F64) < TOL_F64
    assert rel(dx, ref["dx"]).max() < TOL_F64


def test_fp64_single_outputs_match_fused():
    v, x = W.hard_band(2000, seed=203)
    vt, xt = _t(v), _t(x)
    lk, dv, dx = kv.kv_fwd_bwd(vt, xt, bins=64)
    assert torch.equal(kv.kv_log(vt, xt, bins=64), lk)
    assert torch.equal(kv.kv_log_dv(vt, xt, bins=64), dv)
    assert torch.equal(kv.kv_log_dx(vt, xt, bins=64), dx)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_lanes_per_pair(lanes):
    """Splitting a pair's bins over L lanes (shuffle reduction) changes only summation order."""
    v, x = W.full_domain(1000, seed=204)
    ref = oracle.o1(v, x, bins=128, precision="long")
    out = kv.kv_fwd_bwd_ex(_t(v), _t(x), bins=128, lanes=lanes)
    assert rel_logk(_np(out["logk"]), ref["logk"]).max() < TOL_F64
    assert rel(_np(out["dx"]), ref["dx"]).max() < TOL_F64
    outm = kv.kv_fwd_bwd_ex(_t(v, torch.float32), _t(x, torch.float32), bins=32, lanes=lanes)
    ref32 = oracle.o1(v.astype(np.float32), x.astype(np.float32), bins=32, log_eps=MIXED_LOG_EPS,
                      precision="long")
    assert rel_logk(_np(outm["logk"]), ref32["logk"]).max() < TOL_MIXED


def test_analytic_peak_start_flag():
    """KV_FLAG_PEAK_ANALYTIC_START (the FP64 bracket's peak search on [0, asinh(v/x)] instead of
    Algorithm 1's doublings): the FP64 path stays within 1e-13 of the oracle's method (which
    follows Algorithms 1-3), the mixed path with the FP64 bracket within 2e-6, on the whole domain
    and the hard band, including pairs with no peak (v^2 <= x) and edge inputs."""
    v1, x1 = W.full_domain(3000, seed=231)
    v2, x2 = W.hard_band(3000, seed=232)
    v = np.concatenate([v1, v2, [0.0, 1.0, 1e-3, 1000.0, 50.0, -7.5, 2.0]])
    x = np.concatenate([x1, x2, [1.0, 1.0, 1e-6, 1e-6, 1e5, 3.0, 4.0]])
    ref = oracle.o1(v, x, bins=128, precision="long")
    out = kv.kv_fwd_bwd_ex(_t(v), _t(x), bins=128, analytic_peak_start=True)
    assert rel_logk(_np(out["logk"]), ref["logk"]).max() < TOL_F64
    z = v == 0
    assert np.all(_np(out["dv"])[z] == 0)
    assert rel(_np(out["dv"])[~z], ref["dv"][~z]).max() < TOL_F64
    assert rel(_np(out["dx"]), ref["dx"]).max() < TOL_F64
    plain = kv.kv_fwd_bwd_ex(_t(v), _t(x), bins=128)
    assert not torch.equal(plain["logk"], out["logk"])  # the flag reached the kernel
    (vf, v32), (xf, x32) = W.to_f32(v, x)
    ref32 = oracle.o1(v32, x32, bins=32, log_eps=MIXED_LOG_EPS, precision="long")
    o32 = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=32, analytic_peak_start=True)
    assert rel_logk(_np(o32["logk"]), ref32["logk"]).max() < TOL_MIXED
    assert rel(_np(o32["dx"]), ref32["dx"]).max() < TOL_MIXED


@pytest.mark.parametrize("n", [1, 31, 4096, 5000])
def test_fp64_small_batches_every_lane_split(n):
    """Small batches, where every lane brackets its own pair and groups of L lanes then share
    the pairs' bins (constants by warp shuffles): all L give the oracle's results at 1e-13, and
    a ragged last warp stores exactly its pairs."""
    v, x = W.uniform_small(n, seed=233)
    ref = oracle.o1(v, x, bins=128, precision="long")
    for lanes in (1, 4, 32):
        out = kv.kv_fwd_bwd_ex(_t(v), _t(x), bins=128, lanes=lanes)
        assert rel_logk(_np(out["logk"]), ref["logk"]).max() < TOL_F64
        assert rel(_np(out["dx"]), ref["dx"]).max() < TOL_F64


def test_bracket_matches_oracle():
    """kv_bracket (Algorithms 1-3 on the GPU) against the oracle's bracket."""
    v, x = W.full_domain(3000, seed=205)
    t0, tp, t1, G = (_np(t) for t in kv.kv_bracket(_t(v), _t(x)))
    ref = oracle.o1(v, x, precision="long", bracket=True)
    width = ref["t1"] - ref["t0"]
    # the same algorithm: agreement far inside the final FindZero step
    assert np.max(np.abs(t0 - ref["t0"]) / width) < 1e-6
    assert np.max(np.abs(t1 - ref["t1"]) / width) < 1e-6
    assert np.max(np.abs(tp - ref["tp"]) / width) < 1e-6
    assert rel_logk(G, ref["G"]).max() < 1e-13


@pytest.mark.parametrize("n", [0, 1, 31, 33, 129, 4097])
def test_ragged_sizes(n):
    v, x = W.full_domain(max(n, 1), seed=206)
    v, x = v[:n], x[:n]
    lk, dv, dx = kv.kv_fwd_bwd(_t(v), _t(x), bins=64)
    if n == 0:
        assert lk.numel() == 0
        return
    ref = oracle.o1(v, x, bins=64, precision="long")
    assert rel_logk(_np(lk), ref["logk"]).max() < TOL_F64
    assert rel(_np(dx), ref["dx"]).max() < TOL_F64


@pytest.mark.parametrize("bracket", ["plain64", "plain", "f32", "mlp"])
def test_max_bins_every_path(bracket):
    """The largest bin count the boundary accepts (KV_MAX_BINS) on every path: the FP64 bins'
    recurrences (refreshed every 32 steps) and block sums, and the FP32 bins' block-compensated
    sums, keep their accuracy over 4097 bins."""
    v, x = W.full_domain(256, seed=215)
    bins = N.KV_MAX_BINS
    if bracket == "plain64":
        lk, dv, dx = (_np(t) for t in kv.kv_fwd_bwd(_t(v), _t(x), bins=bins))
        ref = oracle.o1(v, x, bins=bins, precision="long")
        tol, v64 = TOL_F64, v
    else:
        (vf, v64), (xf, x64) = W.to_f32(v, x)
        net = learned.default_network(DEV) if bracket == "mlp" else None
        out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=bins, bracket=bracket,
                               mlp=net)
        lk, dv, dx = (_np(out[k]) for k in ("logk", "dv", "dx"))
        ref = oracle.o1(v64, x64, bins=bins, log_eps=MIXED_LOG_EPS, precision="long")
        tol = TOL_MIXED
    assert rel_logk(lk, ref["logk"]).max() < tol
    assert _deriv_ok(dv, ref["dv"], v64, tol) < tol
    assert rel(dx, ref["dx"]).max() < tol


def test_edge_cases_both_paths():
    v = np.array([1.0, 0.0, -2.0, 3.0, -3.0, np.inf, -np.inf, 1.0, np.nan, 1.0, 0.0, -2.5])
    x = np.array([0.0, 0.0, 0.0, np.inf, np.inf, 1.0, 1.0, -1.0, 1.0, np.nan, np.inf, 3.0])
    ref = oracle.o1(v, x, precision="long")
    for dtype in (torch.float64, torch.float32):
        out = kv.kv_fwd_bwd_ex(_t(v, dtype), _t(x, dtype), status=True)
        for k in ("logk", "dv", "dx"):
            g = _np(out[k])
            r = ref[k]
            same = (np.isnan(g) & np.isnan(r)) | (g == r) | (np.isfinite(r) & (np.abs(g - r) <= 1e-5 * np.abs(r)))
            assert same.all(), (dtype, k, g, r)
        st = out["status"].cpu().numpy()
        assert np.all(st[:11] == 1) and st[11] == 0
        assert np.signbit(_np(out["dv"])[4]) and np.signbit(_np(out["dv"])[11])


def test_negative_order_symmetry():
    v, x = W.full_domain(2000, seed=207)
    a = kv.kv_fwd_bwd(_t(v), _t(x))
    b = kv.kv_fwd_bwd(_t(-v), _t(x))
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2]) and torch.equal(a[1], -b[1])


# ------------------------------------------------------------------ mixed path

@pytest.mark.parametrize("bins", [32, 64, 128])
def test_mixed_hard_band_bins_sweep(bins):
    """The 16M-pair workload's recipe (75 % bulk, 25 % |v - x| < 0.1 v), sampled."""
    v, x = W.hard_band(20000, seed=208)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    lk, dv, dx = (_np(t) for t in kv.kv_fwd_bwd(_t(vf, torch.float32), _t(xf, torch.float32), bins=bins))
    ref = oracle.o1(v64, x64, bins=bins, log_eps=MIXED_LOG_EPS, precision="long")
    assert rel_logk(lk, ref["logk"]).max() < TOL_MIXED
    assert _deriv_ok(dv, ref["dv"], v64, TOL_MIXED) < TOL_MIXED
    assert rel(dx, ref["dx"]).max() < TOL_MIXED
    truth = oracle.dense(v64[:3000], x64[:3000])
    assert rel_logk(lk[:3000], truth["logk"]).max() < TOL_MIXED
    assert rel(dx[:3000], truth["dx"]).max() < TOL_MIXED


def test_mixed_full_target_domain():
    """v in [0, 1000], x in [1e-6, 1e5] against the dense-quadrature truth at the default
    40 bins (at 32 bins the trapezoid itself misses 2e-6 in d/dx for small v and x < 1e-4)."""
    v, x = W.full_domain(12000, seed=209)
    v = np.concatenate([v, [0.0, 0.5, 1000.0, 1000.0, 0.0, 999.5, 459.7, 1.47884]])
    x = np.concatenate([x, [1e-6, 1.0, 1e-6, 1e5, 1e5, 3.0, 301.2, 1.52459e-06]])
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    lk, dv, dx = (_np(t) for t in kv.kv_fwd_bwd(_t(vf, torch.float32), _t(xf, torch.float32)))
    truth = oracle.dense(v64, x64)
    assert rel_logk(lk, truth["logk"]).max() < TOL_MIXED
    assert _deriv_ok(dv, truth["dv"], v64, TOL_MIXED) < TOL_MIXED
    assert rel(dx, truth["dx"]).max() < TOL_MIXED


def test_full_size_hard_band_sampled():
    """The full 16,777,216-pair mixed launch (the bench's configuration), checked on 4096
    sampled pairs against the oracle, plus NaN-freeness of every output."""
    n = 16_777_216
    v, x = W.hard_band(n, seed=1)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    vt, xt = _t(vf, torch.float32), _t(xf, torch.float32)
    lk, dv, dx = kv.kv_fwd_bwd(vt, xt, bins=32)
    torch.cuda.synchronize()
    for t in (lk, dv, dx):
        assert torch.isfinite(t).all()
    idx = np.random.default_rng(210).choice(n, 4096, replace=False)
    ref = oracle.o1(v64[idx], x64[idx], bins=32, log_eps=MIXED_LOG_EPS, precision="long")
    assert rel_logk(_np(lk)[idx], ref["logk"]).max() < TOL_MIXED
    assert _deriv_ok(_np(dv)[idx], ref["dv"], v64[idx], TOL_MIXED) < TOL_MIXED
    assert rel(_np(dx)[idx], ref["dx"]).max() < TOL_MIXED
    # and against the integral itself (dense quadrature), on part of the sample
    truth = oracle.dense(v64[idx[:1024]], x64[idx[:1024]])
    assert rel_logk(_np(lk)[idx[:1024]], truth["logk"]).max() < TOL_MIXED
    assert _deriv_ok(_np(dv)[idx[:1024]], truth["dv"], v64[idx[:1024]], TOL_MIXED) < TOL_MIXED
    assert rel(_np(dx)[idx[:1024]], truth["dx"]).max() < TOL_MIXED


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("transfer,pinned", [("auto", False), ("staged", True), ("direct", True), ("auto", True)])
def test_host_buffer_call_matches_device_call(transfer, pinned):
    # pageable buffers take the staged copies; pinned ones either transfer, so every route must
    # give the device call's results bit for bit
    v, x = W.hard_band(5_000_000, seed=211)
    vf = v.astype(np.float32)
    xf = x.astype(np.float32)
    hv, hx = (_pinned(vf), _pinned(xf)) if pinned else (vf, xf)
    out = tuple(_pinned(np.zeros_like(vf)) if pinned else np.zeros_like(vf) for _ in range(3))
    lk_h, dv_h, dx_h = kv.kv_fwd_bwd_host(hv, hx, bins=32, out=out, transfer=transfer)
    lk, dv, dx = kv.kv_fwd_bwd(_t(vf, torch.float32), _t(xf, torch.float32), bins=32)
    assert np.array_equal(lk_h, lk.cpu().numpy())
    assert np.array_equal(dv_h, dv.cpu().numpy())
    assert np.array_equal(dx_h, dx.cpu().numpy())


def test_host_buffer_call_learned_path_direct():
    # the fast path (with its fallback list in device memory) on pinned host buffers in place
    net = learned.default_network(torch.device("cuda", 0))
    v, x = W.hard_band(3_000_001, seed=213)
    vf, xf = v.astype(np.float32), x.astype(np.float32)
    out = tuple(_pinned(np.zeros_like(vf)) for _ in range(3))
    lk_h, dv_h, dx_h = kv.kv_fwd_bwd_host(_pinned(vf), _pinned(xf), bins=32, bracket="mlp", mlp=net,
                                          out=out, transfer="direct")
    r = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=32, bracket="mlp", mlp=net)
    assert np.array_equal(lk_h, r["logk"].cpu().numpy())
    assert np.array_equal(dv_h, r["dv"].cpu().numpy())
    assert np.array_equal(dx_h, r["dx"].cpu().numpy())


def test_host_direct_rejects_unpinned_buffers():
    # the check runs on the host before any launch: pageable memory is not device-addressable
    vf = np.linspace(0.5, 3.0, 1000, dtype=np.float32)
    with pytest.raises(RuntimeError):
        kv.kv_fwd_bwd_host(vf, vf.copy(), bins=32, transfer="direct")
    # one pinned and one pageable input: rejected as well
    with pytest.raises(RuntimeError):
        kv.kv_fwd_bwd_host(_pinned(vf), vf.copy(), bins=32, transfer="direct")
    assert kv.host_direct_supported() in (True, False)


def test_scratch_pool_trim_and_reuse():
    # scratch memory is kept by the library's pool between calls; trimming releases it and the
    # next call allocates again
    v, x = W.hard_band(1 << 20, seed=214)
    vt, xt = _t(v.astype(np.float32), torch.float32), _t(x.astype(np.float32), torch.float32)
    net = learned.default_network(DEV)
    r1 = kv.kv_fwd_bwd_ex(vt, xt, bins=32, bracket="mlp", mlp=net)
    torch.cuda.synchronize()
    kv.trim_memory()
    r2 = kv.kv_fwd_bwd_ex(vt, xt, bins=32, bracket="mlp", mlp=net)
    for k in ("logk", "dv", "dx"):
        assert torch.equal(r1[k], r2[k])
    kv.trim_memory()


# ------------------------------------------------------------------ reductions and autograd

def test_sum_is_deterministic_and_exact_enough():
    a = np.random.default_rng(212).standard_normal(3_000_001)
    t = _t(a)
    s1 = kv.kv_sum(t).item()
    s2 = kv.kv_sum(t).item()
    assert s1 == s2
    assert abs(s1 - np.sum(a, dtype=np.float64)) < 1e-9
    assert kv.kv_sum(_t(np.zeros(0))).item() == 0.0


def test_autograd_gh_loglik_against_oracle_and_fd():
    """Generalized-hyperbolic-style log-likelihood sum_i log K_{lam_i}(x_i) in float32: the
    gradient through the fused backward against the oracle's derivatives and central finite
    differences (h = 1e-4) of the oracle."""
    lam, x, alpha, delta, z = W.gh_likelihood(50_000, seed=2)
    lt = _t(lam, torch.float32).requires_grad_(True)
    xt = _t(x, torch.float32).requires_grad_(True)
    loss = kv.kv_sum(kv.log_besselk(lt, xt, bins=32))
    lk = kv.log_besselk(lt, xt, bins=32)
    lk.backward(torch.ones_like(lk))
    l64, x64 = lam.astype(np.float64), x.astype(np.float64)
    ref = oracle.o1(l64, x64, bins=32, log_eps=MIXED_LOG_EPS, precision="long")
    assert abs(loss.item() - ref["logk"].sum()) < 2e-6 * np.abs(ref["logk"]).sum()
    assert _deriv_ok(_np(lt.grad), ref["dv"], l64, TOL_MIXED) < TOL_MIXED
    assert rel(_np(xt.grad), ref["dx"]).max() < TOL_MIXED
    # central finite differences of the FP64 oracle on a subsample
    k = slice(0, 500)
    h = 1e-4
    fd_v = (oracle.o1(l64[k] + h, x64[k], precision="long")["logk"]
            - oracle.o1(l64[k] - h, x64[k], precision="long")["logk"]) / (2 * h)
    fd_x = (oracle.o1(l64[k], x64[k] + h, precision="long")["logk"]
            - oracle.o1(l64[k], x64[k] - h, precision="long")["logk"]) / (2 * h)
    gv = _np(lt.grad)[k]
    gx = _np(xt.grad)[k]
    # FD truncation error is O(h^2 |f'''|): compare with a tolerance that covers it
    assert np.max(np.abs(gv - fd_v) / np.maximum(1, np.abs(fd_v))) < 1e-4
    assert np.max(np.abs(gx - fd_x) / np.maximum(1, np.abs(fd_x))) < 1e-4
    # chain rule to the distribution parameters: x = delta * alpha * sqrt(1 + z^2)
    gal = float((xt.grad.double() * _t(delta * np.sqrt(1 + z.astype(np.float64) ** 2))).sum())
    gal_ref = float((ref["dx"] * delta * np.sqrt(1 + z.astype(np.float64) ** 2)).sum())
    assert abs(gal - gal_ref) < 1e-5 * np.abs(ref["dx"] * delta).sum()


def test_fused_grad_out_epilogue():
    v, x = W.full_domain(3000, seed=213)
    go = np.random.default_rng(214).standard_normal(3000)
    out = kv.kv_fwd_bwd_ex(_t(v), _t(x), bins=128, grad_out=_t(go))
    ref = kv.kv_fwd_bwd(_t(v), _t(x), bins=128)
    assert torch.equal(out["logk"], ref[0])
    assert torch.allclose(out["dv"], ref[1] * _t(go), rtol=1e-15, atol=0)
    assert torch.allclose(out["dx"], ref[2] * _t(go), rtol=1e-15, atol=0)
