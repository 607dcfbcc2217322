"""The learned bracket on the GPU: training kernels against the MLP oracle, checkpoints, and the
fast path (MLP bracket, float-float offset, FP32 bins, plain fallback) against the method oracle.
"""
import os
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
from conftest import rel, rel_logk
from oracle import mlp as omlp
from paper_2108_11560_gb300 import _native as N
from paper_2108_11560_gb300 import kv, learned
from paper_2108_11560_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TOL = 2e-6
LOG_EPS = -20.0


def _t(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _synthetic_targets(v, x, seed):
    """A bracket around the exact peak with random widths (any targets serve a gradient check)."""
    rng = np.random.default_rng(seed)
    tp = omlp.peak(v, x)
    t0 = np.maximum(tp - rng.uniform(0.01, 2.0, v.size), 0.0)
    t1 = tp + rng.uniform(0.01, 4.0, v.size)
    return t0, t1


@pytest.fixture(scope="module")
def net():
    return learned.default_network(DEV)


def test_loss_and_gradient_match_oracle():
    v, x = W.learned_bracket(3000, seed=301)
    v = v.astype(np.float32).astype(np.float64)
    x = x.astype(np.float32).astype(np.float64)
    t0, t1 = _synthetic_targets(v, x, 302)
    p = np.random.default_rng(303).normal(0, 0.2, N.KV_MLP_NPARAMS).astype(np.float32)
    m = learned.Mlp.create(0)
    m.set_params(p)
    assert np.array_equal(m.params(), p)
    loss, g = m.loss_grad(_t(v), _t(x), _t(t0), _t(t1))
    ref_loss, ref_g = omlp.loss_grad(p.astype(np.float64), v, x, t0, omlp.peak(v, x), t1)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))


def test_adam_steps_match_oracle():
    """Five Adam steps through the library's kernels (same SplitMix64 batches) against the
    oracle's training loop."""
    v, x = W.learned_bracket(4096, seed=304)
    v = v.astype(np.float32).astype(np.float64)
    x = x.astype(np.float32).astype(np.float64)
    t0, t1 = _synthetic_targets(v, x, 305)
    p = np.random.default_rng(306).normal(0, 0.2, N.KV_MLP_NPARAMS).astype(np.float32)
    m = learned.Mlp.create(0)
    m.set_params(p)
    lr = 1e-3
    losses = m.train(_t(v), _t(x), _t(t0), _t(t1), steps=5, batch=512, lr=lr, seed=7)
    ref_p, ref_losses = omlp.train(p.astype(np.float64), v, x, t0, t1, steps=5, batch=512, lr=lr,
                                   beta1=0.9, beta2=0.999, eps=1e-8, seed=7)
    assert np.allclose(losses, ref_losses, rtol=1e-4)
    d = np.abs(m.params() - ref_p)
    # Adam normalises each step to about lr: agreement far below lr except where a gradient
    # component is at rounding level and its sign is arbitrary
    assert np.quantile(d, 0.99) < 0.01 * lr
    assert d.max() < 10 * lr


def test_fast_path_sees_trained_weights(net):
    """The fast path reads the small layers' weights from a host copy of the parameters: after
    training steps on the device, its results equal those of a fresh handle given the trained
    parameters (and differ from the untrained ones)."""
    v, x = W.hard_band(50000, seed=312)
    vf, xf = _t(v, torch.float32), _t(x, torch.float32)
    m = learned.Mlp.create(0)
    m.set_params(net.params())
    before = kv.kv_fwd_bwd_ex(vf, xf, bins=32, bracket="mlp", mlp=m, status=True)
    tv, tx, t0, t1 = learned.training_set(DEV, n=8192, seed=313)
    m.train(tv, tx, t0, t1, steps=20, batch=1024, lr=1e-2, seed=3)
    after = kv.kv_fwd_bwd_ex(vf, xf, bins=32, bracket="mlp", mlp=m, status=True)
    fresh = learned.Mlp.create(0)
    fresh.set_params(m.params())
    ref = kv.kv_fwd_bwd_ex(vf, xf, bins=32, bracket="mlp", mlp=fresh, status=True)
    for k in ("logk", "dv", "dx", "status"):
        assert torch.equal(after[k], ref[k]), k
    assert not torch.equal(after["status"], before["status"]) or not torch.equal(after["logk"], before["logk"])


def test_checkpoint_roundtrip(net):
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "net.kvmlp")
        net.save(path)
        back = learned.Mlp.load(path)
        assert np.array_equal(back.params(), net.params())
        v, x = W.learned_bracket(1000, seed=307)
        vf, xf = _t(v, torch.float32), _t(x, torch.float32)
        a0, a1 = net.predict(vf, xf)
        b0, b1 = back.predict(vf, xf)
        assert torch.equal(a0, b0) and torch.equal(a1, b1)
        with open(path, "r+b") as f:
            f.write(b"XXXXXXXX")
        with pytest.raises(N.KvError):
            learned.Mlp.load(path)


def test_predictions_match_oracle_forward(net):
    """The inference kernel (BF16 W2 and hidden units, FP32 accumulation) against the oracle's
    float64 forward pass on the same FP32 parameters, in the log half-widths."""
    v, x = W.learned_bracket(4000, seed=308)
    v = v.astype(np.float32).astype(np.float64)
    x = x.astype(np.float32).astype(np.float64)
    t0, t1 = net.predict(_t(v, torch.float32), _t(x, torch.float32))
    tp = omlp.peak(v, x)
    params = net.params().astype(np.float64)
    r0, r1 = omlp.predict(params, v, x, tp)
    # the BF16 rounding of W2 and of h1 (each within 2^-9 relative) moves hidden unit j by at
    # most 2^-8 sum_i |W2_ji| |h1_i|, and output k by at most sum_j |W3_kj| times that
    P = omlp.unpack(params)
    h1 = omlp.forward(params, v, x)["h1"]
    dz2 = 1.01 * 2.0 ** -8 * (h1 @ np.abs(P["W2"]).T)
    bound = dz2 @ np.abs(P["W3"]).T  # [n, 2] in the network's output units
    L = lambda a: np.log(np.maximum(a, 0) + omlp.DELTA)
    e1 = np.abs(L(_np(t1) - tp) - L(r1 - tp))
    assert np.all(e1 <= omlp.OUT_SCALE[2] * bound[:, 1] + 2e-3)
    sel = (_np(t0) > 0) & (r0 > 0)  # both sides unclamped
    e0 = np.abs(L(tp[sel] - _np(t0)[sel]) - L(tp[sel] - r0[sel]))
    assert np.all(e0 <= omlp.OUT_SCALE[0] * bound[sel, 0] + 2e-3)


def test_trained_network_fits_its_targets(net):
    """After training, the predicted log half-widths are within a few percent of the plain
    bracket's on fresh pairs of the training distribution."""
    v, x, t0, t1 = learned.training_set(DEV, n=20000, seed=309)
    p0, p1 = net.predict(v.float(), x.float())
    tp = omlp.peak(_np(v), _np(x))
    L = lambda a: np.log(np.maximum(a, 0) + omlp.DELTA)
    e1 = np.abs(L(_np(p1) - tp) - L(_np(t1) - tp))
    assert np.median(e1) < 0.03 and np.quantile(e1, 0.99) < 0.2


@pytest.mark.parametrize("bins", [32, 40, 41])
def test_mlp_path_matches_oracle(net, bins):
    """The fast path on the hard-band and learned-bracket workloads against the oracle's method
    (FP64 ... long double) and the dense truth; every pair, fallback or not."""
    v1, x1 = W.hard_band(20000, seed=310)
    v2, x2 = W.learned_bracket(20000, seed=311)
    v = np.concatenate([v1, v2, [0.0, 0.5, 200.0, 3.0]])
    x = np.concatenate([x1, x2, [1e-4, 1.0, 1e-4, 1e4]])
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    fb = torch.zeros(1, dtype=torch.int64, device=DEV)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=bins, bracket="mlp",
                           mlp=net, status=True, fallback_count=fb)
    lk, dv, dx = _np(out["logk"]), _np(out["dv"]), _np(out["dx"])
    st = out["status"].cpu().numpy()
    ref = oracle.o1(v64, x64, bins=bins, log_eps=LOG_EPS, precision="long")
    assert rel_logk(lk, ref["logk"]).max() < TOL
    z = v64 == 0
    assert np.all(dv[z] == 0)
    assert rel(dv[~z], ref["dv"][~z]).max() < TOL
    assert rel(dx, ref["dx"]).max() < TOL
    n_fb = int(np.count_nonzero(st & N.KV_PAIR_FALLBACK))
    assert fb.item() == n_fb
    assert n_fb < 0.02 * v.size, n_fb / v.size
    truth = oracle.dense(v64[::10], x64[::10])
    assert rel_logk(lk[::10], truth["logk"]).max() < TOL
    assert rel(dx[::10], truth["dx"]).max() < TOL


@pytest.mark.parametrize("bins", [32, 64])
def test_mlp_path_coarse_eps(net, bins):
    """At log eps = -11 (window [-23, -11]) the network's ends, trained for e^-26, lie outside the
    window for most pairs, so the check's Newton corrections run, and bin n is one of the bins
    (its terms are not taken from the check above log eps = -12).  The oracle's method itself is
    then only within its truncation error of the dense truth: the fast path must stay within three
    times the method's largest error at the same eps plus the mixed tolerance."""
    le = -11.0
    v, x = W.hard_band(6000, seed=330)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=bins, bracket="mlp",
                           mlp=net, log_eps=le, status=True)
    lk, dv, dx = _np(out["logk"]), _np(out["dv"]), _np(out["dx"])
    st = out["status"].cpu().numpy()
    assert np.all(np.isfinite(lk)) and np.all(np.isfinite(dx))
    truth = oracle.dense(v64, x64)
    ref = oracle.o1(v64, x64, bins=bins, log_eps=le, precision="long")
    z = v64 == 0
    for name, got in (("logk", lk), ("dv", dv), ("dx", dx)):
        e = rel_logk if name == "logk" else rel
        keep = ~z if name == "dv" else np.ones(v.size, bool)
        method = e(ref[name][keep], truth[name][keep]).max()
        assert e(got[keep], truth[name][keep]).max() < 3 * method + TOL, (name, method)
    assert np.all(dv[z] == 0)
    assert np.count_nonzero(st & N.KV_PAIR_FALLBACK) < 0.05 * v.size


@pytest.mark.parametrize("bins", [2, 4, 5, 7, 8, 33, 44])
def test_end_terms_from_the_check(net, bins):
    """Bin n's trapezoid terms taken from the range check's evaluation of the right end (the
    default, from 4 bins up) against bin n computed as one of the bins, on the same learned ranges:
    the two agree to FP32 rounding, including bin counts that leave a scalar tail of bins and the
    compensated instance (44 bins)."""
    v, x = W.hard_band(20000, seed=331)
    (vf, _), (xf, _) = W.to_f32(v, x)
    vt, xt = _t(vf, torch.float32), _t(xf, torch.float32)
    on = kv.kv_fwd_bwd_ex(vt, xt, bins=bins, bracket="mlp", mlp=net, status=True)
    prev = kv.debug_set_end_terms(False)
    try:
        off = kv.kv_fwd_bwd_ex(vt, xt, bins=bins, bracket="mlp", mlp=net, status=True)
    finally:
        kv.debug_set_end_terms(True)
    assert prev == 1
    assert torch.equal(on["status"], off["status"])  # the same ranges
    assert rel_logk(_np(on["logk"]), _np(off["logk"])).max() < 5e-7
    assert rel(_np(on["dv"]), _np(off["dv"])).max() < 1e-6
    assert rel(_np(on["dx"]), _np(off["dx"])).max() < 1e-6


def test_fallback_path_is_exact_enough():
    """A network whose outputs are NaN fails every check and sends every pair to the
    plain-bracket fallback, whose results still meet the tolerance; an untrained network is
    rescued in part by the end corrections."""
    bad = learned.Mlp.create(5)
    p = bad.params()
    p[-2:] = np.nan  # b3: both outputs NaN
    bad.set_params(p)
    v, x = W.hard_band(8000, seed=312)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    fb = torch.zeros(1, dtype=torch.int64, device=DEV)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=32, bracket="mlp",
                           mlp=bad, status=True, fallback_count=fb)
    st = out["status"].cpu().numpy()
    assert fb.item() == np.count_nonzero(st & N.KV_PAIR_FALLBACK) == v.size
    ref = oracle.o1(v64, x64, bins=32, log_eps=LOG_EPS, precision="long")
    assert rel_logk(_np(out["logk"]), ref["logk"]).max() < TOL
    assert rel(_np(out["dx"]), ref["dx"]).max() < TOL
    untrained = learned.Mlp.create(6)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=32, bracket="mlp",
                           mlp=untrained, status=True)
    assert rel_logk(_np(out["logk"]), ref["logk"]).max() < TOL
    assert rel(_np(out["dx"]), ref["dx"]).max() < TOL


def test_mlp_path_edge_cases(net):
    v = np.array([1.0, 0.0, -2.0, 3.0, -3.0, np.inf, -np.inf, 1.0, np.nan, 1.0, 0.0, -2.5])
    x = np.array([0.0, 0.0, 0.0, np.inf, np.inf, 1.0, 1.0, -1.0, 1.0, np.nan, np.inf, 3.0])
    out = kv.kv_fwd_bwd_ex(_t(v, torch.float32), _t(x, torch.float32), bracket="mlp", mlp=net,
                           status=True)
    ref = oracle.o1(v, x, precision="long")
    for k in ("logk", "dv", "dx"):
        g = _np(out[k])
        r = ref[k]
        both_nan = np.isnan(g) & np.isnan(r)
        close = np.isfinite(r) & (np.abs(g - np.nan_to_num(r)) <= 2e-6 * np.maximum(1, np.abs(np.nan_to_num(r))))
        assert np.all(both_nan | (g == r) | close), (k, g, r)
    st = out["status"].cpu().numpy()
    assert np.all(st[:11] == N.KV_PAIR_EDGE) and not (st[11] & N.KV_PAIR_EDGE)


@pytest.mark.parametrize("second", [False, True])
def test_tensor_core_wait_running_out_falls_back(net, second):
    """Failure handling of the fast path, with no fault: with the wait for the tensor-core results
    limited to zero tries, every CTA gives up at its first tile and hands all its pairs, edge pairs
    included, to the fallback pass.  The outputs must still match the oracle (edge pairs: exactly
    what the normal call gives), every regular pair carries the fallback bit, and the next call
    with the default limit runs normally on the same context."""
    v1, x1 = W.hard_band(50_000, seed=316)
    ve = np.array([1.0, 0.0, -2.0, 3.0, np.inf, 1.0, np.nan, 1.0, -2.5])
    xe = np.array([0.0, 0.0, np.inf, np.inf, 1.0, -1.0, 1.0, np.nan, 3.0])
    v = np.concatenate([v1[:25_000], ve, v1[25_000:]])
    x = np.concatenate([x1[:25_000], xe, x1[25_000:]])
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    edge = np.isnan(vf) | np.isnan(xf) | (xf <= 0) | np.isinf(xf) | np.isinf(vf)
    vt, xt = _t(vf, torch.float32), _t(xf, torch.float32)
    fb = torch.zeros(1, dtype=torch.int64, device=DEV)
    prev = kv.debug_set_wait_limit(0)
    try:
        out = kv.kv_fwd_bwd_ex(vt, xt, bins=40, bracket="mlp", mlp=net, status=True, fallback_count=fb,
                               second=second)
        torch.cuda.synchronize()
    finally:
        kv.debug_set_wait_limit(prev)
    assert prev == -1
    st = out["status"].cpu().numpy()
    assert np.all(st[edge] == N.KV_PAIR_EDGE)
    assert np.all(st[~edge] & N.KV_PAIR_FALLBACK)
    assert fb.item() == v.size  # every pair was handed over
    fb2 = torch.zeros(1, dtype=torch.int64, device=DEV)
    normal = kv.kv_fwd_bwd_ex(vt, xt, bins=40, bracket="mlp", mlp=net, status=True, fallback_count=fb2,
                              second=second)
    assert fb2.item() < 0.02 * v.size
    keys = ("logk", "dv", "dx") + (("d2v", "dvx", "d2x") if second else ())
    for k in keys:
        assert np.array_equal(_np(out[k])[edge], _np(normal[k])[edge], equal_nan=True), k
    fin = ~edge
    ref = oracle.o1(v64[fin], x64[fin], bins=40, log_eps=LOG_EPS, precision="long", second=second)
    assert rel_logk(_np(out["logk"])[fin], ref["logk"]).max() < TOL
    dv = _np(out["dv"])[fin]
    z = v64[fin] == 0
    assert np.all(dv[z] == 0)
    assert rel(dv[~z], ref["dv"][~z]).max() < TOL
    assert rel(_np(out["dx"])[fin], ref["dx"]).max() < TOL
    if second:
        scale = {"d2v": ref["dv"] ** 2 + np.abs(ref["d2v"]), "d2x": ref["dx"] ** 2 + np.abs(ref["d2x"]),
                 "dvx": np.abs(ref["dv"] * ref["dx"]) + np.abs(ref["dvx"])}
        for k in ("d2v", "dvx", "d2x"):
            g = _np(out[k])[fin]
            nz = scale[k] > 0
            assert (np.abs(g[nz] - ref[k][nz]) / scale[k][nz]).max() < TOL, k


@pytest.mark.parametrize("n", [0, 1, 127, 129, 1_000_003])
def test_mlp_path_ragged_sizes(net, n):
    """Tiles of 128 pairs per CTA and a persistent grid: a size below one tile, around one tile,
    and a large size with a ragged last tile, against the oracle's method (sampled)."""
    v, x = W.hard_band(max(n, 1), seed=317)
    (vf, v64), (xf, x64) = W.to_f32(v[:n], x[:n])
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=32, bracket="mlp", mlp=net)
    if n == 0:
        assert out["logk"].numel() == 0
        return
    idx = np.unique(np.concatenate([np.arange(min(n, 256)), np.arange(max(n - 256, 0), n),
                                    np.random.default_rng(318).choice(n, min(n, 2000), replace=False)]))
    ref = oracle.o1(v64[idx], x64[idx], bins=32, log_eps=LOG_EPS, precision="long")
    assert rel_logk(_np(out["logk"])[idx], ref["logk"]).max() < TOL
    z = v64[idx] == 0
    assert rel(_np(out["dv"])[idx][~z], ref["dv"][~z]).max() < TOL
    assert rel(_np(out["dx"])[idx], ref["dx"]).max() < TOL


def test_mlp_path_full_size_sampled(net):
    """The bench's launch: 16,777,216 hard-band pairs, fast path at 32 bins, sampled check."""
    n = 16_777_216
    v, x = W.hard_band(n, seed=1)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    fb = torch.zeros(1, dtype=torch.int64, device=DEV)
    out = kv.kv_fwd_bwd_ex(_t(vf, torch.float32), _t(xf, torch.float32), bins=32, bracket="mlp",
                           mlp=net, fallback_count=fb)
    for k in ("logk", "dv", "dx"):
        assert torch.isfinite(out[k]).all()
    assert fb.item() < 0.01 * n
    idx = np.random.default_rng(313).choice(n, 4096, replace=False)
    ref = oracle.o1(v64[idx], x64[idx], bins=32, log_eps=LOG_EPS, precision="long")
    assert rel_logk(_np(out["logk"])[idx], ref["logk"]).max() < TOL
    assert rel(_np(out["dx"])[idx], ref["dx"]).max() < TOL
    z = v64[idx] == 0
    assert rel(_np(out["dv"])[idx][~z], ref["dv"][~z]).max() < TOL


def test_learned_bracket_gain(net):
    """What the trained network gains over the method without it, on the same 4M hard-band pairs
    at 32 bins and the same accuracy bar: against the mixed path with the paper's FP64 bracket,
    and against the fastest form of the method without a network, Algorithms 1-3 in FP32 with the
    same offset, bins and finish (KV_BRACKET_PLAIN_F32).  Both brackets' results are checked
    against the oracle on a sample here as well, so the times compare equal accuracy."""
    n = 1 << 22
    v, x = W.hard_band(n, seed=314)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    vt, xt = _t(vf, torch.float32), _t(xf, torch.float32)

    def timed(**kw):
        out = kv.kv_fwd_bwd_ex(vt, xt, bins=32, **kw)
        for _ in range(2):
            kv.kv_fwd_bwd_ex(vt, xt, bins=32, out=out, **kw)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(5):
            kv.kv_fwd_bwd_ex(vt, xt, bins=32, out=out, **kw)
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 5e3, out

    t_plain, _ = timed(bracket="plain")
    t_f32, o_f32 = timed(bracket="f32")
    t_mlp, o_mlp = timed(bracket="mlp", mlp=net)
    idx = np.random.default_rng(315).choice(n, 2048, replace=False)
    ref = oracle.o1(v64[idx], x64[idx], bins=32, log_eps=LOG_EPS, precision="long")
    for o in (o_f32, o_mlp):
        assert rel_logk(_np(o["logk"])[idx], ref["logk"]).max() < TOL
        assert rel(_np(o["dx"])[idx], ref["dx"]).max() < TOL
    print(f"FP64 bracket {n / t_plain:.3e} pairs/s, FP32 bracket {n / t_f32:.3e} pairs/s, "
          f"learned bracket {n / t_mlp:.3e} pairs/s ({t_f32 / t_mlp:.2f}x the FP32 bracket)")
    assert t_mlp < 0.5 * t_plain
    assert t_mlp * 1.5 < t_f32
