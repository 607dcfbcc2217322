"""bench.py on the CPU: it imports, and its baseline arm (the oracle) prints the contract's JSON
line with the keys the driver reads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_module_imports_and_defines_counts():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.FP32_OPS_PER_BIN > 0 and bench.FP32_OPS_PER_PAIR > 0
    # the instance with plain block sums below the threshold, compensated sums above it
    # bins 0..n-1 run in the bin loop (bin n's terms come from the range check)
    assert bench.fp32_ops(bench.PLAIN_SUMS_MAX_BINS) == bench.FP32_OPS_PER_PAIR + bench.PLAIN_SUMS_MAX_BINS * bench.FP32_OPS_PER_BIN
    assert bench.fp32_ops(64) == bench.FP32_OPS_PER_PAIR_COMP + 64 * bench.FP32_OPS_PER_BIN_COMP
    assert callable(bench._env_rank) and callable(bench.all_reduce_scalar)
    # the SFU figure of a 16.7M-pair step at 32 bins, 0.967 ms, 152 SMs at 2070 MHz
    s = bench.sfu_utilisation(16_777_216, 32, 0.967, 152, 2070.0)
    assert set(s) >= {"achieved", "peak", "unit", "frac", "peak_source"}
    assert abs(s["peak"] - 152 * 32 * 2070e6 / 1e12) < 1e-9
    assert 0.2 < s["frac"] < 0.35 and abs(s["frac"] - s["achieved"] / s["peak"]) < 1e-12
    # issue slots: one warp instruction per sub-partition per clock
    q = bench.issue_utilisation(16_777_216, 32, 0.967, 152, 2070.0)
    assert abs(q["peak"] - 152 * 4 * 2070e6 / 1e12) < 1e-9
    assert 0.5 < q["frac"] < 1.0 and q["inst_per_pair"] == bench.INST_PER_PAIR + 32 * bench.INST_PER_BIN


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_own_arm_fails_loudly_without_a_gpu():
    """No CPU fallback: without a GPU the bench's own arm exits non-zero and prints no result."""
    import pytest

    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode != 0
    assert not any(l.strip().startswith("{") for l in r.stdout.splitlines())


def test_accuracy_certificate_catches_a_wrong_output():
    """The bench's accuracy check (run after the timed steps on the GPU outputs) on CPU tensors:
    outputs equal to the oracle's method pass, and one output moved by 1e-5 relative fails."""
    import numpy as np
    import pytest

    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2108_11560_gb300 import workloads as W

    v, x = W.hard_band(3000, seed=41)
    (vf, v64), (xf, x64) = W.to_f32(v, x)
    v64[5] = 0.0
    ref = oracle.o1(v64, x64, bins=32, log_eps=bench.MIXED_LOG_EPS, precision="long")
    outs = {k: torch.tensor(ref[k], dtype=torch.float64) for k in ("logk", "dv", "dx")}
    idx = bench.sample_indices(v64.size, 500, 3, extra=[7, 2999])
    assert idx[0] == 0 and idx[-1] == v64.size - 1 and 7 in idx and 5 in idx
    assert np.all(np.diff(idx) > 0)
    a = bench.accuracy(outs, v64, x64, idx, 32, bench.MIXED_LOG_EPS, bench.TOL_MIXED)
    assert a["ok"] and a["max_rel_logk"] < 1e-15 and a["pairs"] == idx.size
    go = torch.full((v64.size,), 2.0, dtype=torch.float64)
    scaled = dict(outs, dv=outs["dv"] * 2.0, dx=outs["dx"] * 2.0)
    assert bench.accuracy(scaled, v64, x64, idx, 32, bench.MIXED_LOG_EPS, bench.TOL_MIXED, grad_out=go)["ok"]
    bad = {k: t.clone() for k, t in outs.items()}
    bad["dx"][7] *= 1.0 + 1e-5
    b = bench.accuracy(bad, v64, x64, idx, 32, bench.MIXED_LOG_EPS, bench.TOL_MIXED)
    assert not b["ok"] and 9e-6 < b["max_rel_dx"] < 1.1e-5
    bad = {k: t.clone() for k, t in outs.items()}
    bad["dv"][5] = 1e-30  # d/dv must be exactly 0 at v = 0
    assert not bench.accuracy(bad, v64, x64, idx, 32, bench.MIXED_LOG_EPS, bench.TOL_MIXED)["ok"]


def test_counts_source_hash_is_current_or_flagged():
    """The ncu-derived operation counts are tied to the fast kernel's sources by a hash; the
    bench reports whether they match (a stale count is reported as such, never silently)."""
    sys.path.insert(0, ROOT)
    import bench

    h = bench.counts_source_sha()
    assert isinstance(h, str) and len(h) == 16
    assert isinstance(bench.COUNTS_SOURCE_SHA, str) and len(bench.COUNTS_SOURCE_SHA) == 16


def test_plain_sums_threshold_matches_the_kernels():
    """The bench picks the operation counts of the kernel instance that runs: its threshold must
    be the kernels' own (kPlainSumsMaxBins in kv_bins.cuh)."""
    import re

    sys.path.insert(0, ROOT)
    import bench

    with open(os.path.join(ROOT, "paper_2108_11560_gb300", "csrc", "kv_bins.cuh")) as f:
        m = re.search(r"constexpr int kPlainSumsMaxBins = (\d+);", f.read())
    assert m and int(m.group(1)) == bench.PLAIN_SUMS_MAX_BINS


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the multi-GPU contract launches it (torchrun, two ranks): rank 0 alone runs the
    oracle arm and prints its one line, the other rank exits 0 without work."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port),
                        os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
