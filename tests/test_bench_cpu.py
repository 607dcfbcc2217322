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
    assert callable(bench._env_rank) and callable(bench.all_reduce_scalar)
    # the SFU figure of the 16.7M-pair step at 32 bins, 1.273 ms, 152 SMs at 2070 MHz
    s = bench.sfu_utilisation(16_777_216, 32, 1.273, 152, 2070.0)
    assert set(s) >= {"achieved", "peak", "unit", "frac", "peak_source"}
    assert abs(s["peak"] - 152 * 32 * 2070e6 / 1e12) < 1e-9
    assert 0.2 < s["frac"] < 0.25 and abs(s["frac"] - s["achieved"] / s["peak"]) < 1e-12


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
