"""Throughput of batched log K_v(x) + d/dv + d/dx (pairs/s) on GB300.

One step = one pass of the whole hot path over the 16,777,216-pair hard-band workload
(75 % v ~ U[0, 50], x log-uniform in [1e-3, 1e3]; 25 % |v - x| < 0.1 v), float32 I/O, mixed path:
bracket (learned MLP with plain fallback, or the plain FP64 bracket), FP32 peak-relative bins,
log K, d/dv, d/dx, and the backward epilogue (the derivatives multiplied by an incoming
gradient).  Inputs are resident in HBM before timing; the working set (134 MB in, 201 MB out) is
larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--bins 32] [--bracket mlp|plain]
    python bench.py --impl reference ...   # the CPU oracle on the host cores (baseline arm)

Under torchrun each rank runs its own replica of the workload (pairs are independent: weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2108_11560_gb300 import workloads as W  # noqa: E402
from paper_2108_11560_gb300.distributed import all_reduce_scalar  # noqa: E402
from paper_2108_11560_gb300.distributed import env_rank as _env_rank  # noqa: E402

METRIC = "(v,x) pairs/s for log K_v(x)+∂v+∂x at ≤2e-6 rel err; % of FP32/SFU peak"
UNIT = "pairs/s"
N_PAIRS = 16_777_216
WORKLOAD = "hard_band_16M"
MIXED_LOG_EPS = -20.0

# Algorithmic FP32 work of the learned-bracket fast path, counted operation by operation from
# its formulas with an FMA as one operation and a paired (f32x2) instruction as two:
#   per bin: the abscissa 1, the exponent's x-part (the phi polynomials or e^{+-s}) 15, the rest
#            of the weight 5, the two derivative integrands 7 (+ the tanh polynomial in the ~33 %
#            of warp-blocks that need it, ~2.7), three block-compensated sums 5.25
#                                                                               -> 36 (+ 4 MUFU)
#   per pair: layer 1 and layer 3 on the CUDA cores 256 (layer 2 runs on the tensor cores and
#             is not counted), peak Newton, offset constants, endpoint check, setup and finish
#             ~250                                                              -> 505
# ncu's executed FFMA + FADD + FMUL (+ 2 x FFMA2/FADD2/FMUL2) counters over 4M pairs at 1 and 32
# bins give 35.92 per bin and 505.1 per pair (profiles/kv_mlp_tc_kernel_hard_band_4M.md).
FP32_OPS_PER_BIN = 35.92
MUFU_OPS_PER_BIN = 4
FP32_OPS_PER_PAIR = 505.1
# XU-pipe (MUFU) operations per pair outside the bins, from the same captures
# (smsp__inst_executed_pipe_xu: 46.5 per pair at 1 bin, 4.0 per bin), and the XU pipe's lanes per
# SM per clock that ncu's XU percentages are taken against (170.5 operations per pair in 0.330 ms
# per 4M pairs read as 23.2 % there).
MUFU_OPS_PER_PAIR = 38.5
XU_LANES_PER_SM = 32
# DRAM bytes per pair of the fast-path kernel, from one ncu capture (50.39 MB read + 4.96 MB
# written for 4,194,304 pairs; profiles/kv_mlp_tc_kernel_hard_band_4M.md), scaled to a launch.
# Set to None whenever the kernel changes until it is captured again.
TRAFFIC_BYTES_PER_PAIR = (50.386688e6 + 4.958464e6) / 4194304


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return None
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_baseline(v, x, bins, seconds_target=15.0):
    """The oracle's FP64 fixed-bin method (same bins and eps) on the host cores, on a bounded
    sample of the same workload: its first pairs, sized to about seconds_target of work."""
    import oracle

    oracle.build()
    cores = oracle.host_cores()
    probe = 65536
    t = time.perf_counter()
    oracle.o1(v[:probe], x[:probe], bins=bins, log_eps=MIXED_LOG_EPS)
    rate = probe / (time.perf_counter() - t)
    m = int(min(len(v), max(probe, rate * seconds_target)))
    t = time.perf_counter()
    oracle.o1(v[:m], x[:m], bins=bins, log_eps=MIXED_LOG_EPS)
    dt = time.perf_counter() - t
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {m} pairs of the {WORKLOAD} workload (FP64 fixed-bin method, "
                      f"{bins} bins, eps e^-20), {dt:.1f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle, timed per step on a bounded sample of the workload."""
    rank, _, world = _env_rank()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    v, x = W.hard_band(N_PAIRS, seed=1)
    v = v.astype(np.float32).astype(np.float64)
    x = x.astype(np.float32).astype(np.float64)
    per_step = 262_144
    times = []
    for k in range(args.warmup + args.steps):
        off = (k * per_step) % (N_PAIRS - per_step)
        t = time.perf_counter()
        oracle.o1(v[off:off + per_step], x[off:off + per_step], bins=args.bins, log_eps=MIXED_LOG_EPS)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    total = sum(times)
    val = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs": N_PAIRS, "bins": args.bins,
                   "sample_pairs_per_step": per_step},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.host_cores(), "kind": "oracle",
                         "sample": f"{per_step} consecutive pairs of the {WORKLOAD} workload per step"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def sfu_utilisation(n_pairs, bins, launch_ms, sms, sm_mhz):
    """XU (MUFU: ex2, lg2, rcp) operations per second of the fast-path kernel against the XU
    pipe's peak, the second half of the metric's "% of FP32/SFU peak"."""
    ops = n_pairs * (MUFU_OPS_PER_PAIR + (bins + 1) * MUFU_OPS_PER_BIN)
    achieved = ops / (launch_ms / 1e3)
    peak = sms * XU_LANES_PER_SM * sm_mhz * 1e6
    return {"achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T XU ops/s",
            "frac": achieved / peak,
            "peak_source": f"{sms} SMs x {XU_LANES_PER_SM} XU lanes x {sm_mhz:.0f} MHz (the XU-pipe peak "
                           f"ncu's pipe percentages use)"}


def end_to_end(args, vf, xf, mlp, dist, dev, world):
    """The same call through the host-buffer entry point on pinned host buffers, inside the timed
    region (wall clock around the blocking call): the inputs cross to the GPU and the results
    come back every step, either staged through device buffers by copies or read and written
    in place by the kernels over a coherent CPU-GPU link (transfer "auto" picks)."""
    import torch

    from paper_2108_11560_gb300 import kv

    n = vf.size
    hv = torch.from_numpy(vf).pin_memory().numpy()
    hx = torch.from_numpy(xf).pin_memory().numpy()
    hout = tuple(torch.empty(n, dtype=torch.float32).pin_memory().numpy() for _ in range(3))
    steps = max(3, min(args.steps, 5))
    kw = dict(bins=args.bins, bracket=args.bracket, mlp=mlp, out=hout, transfer=args.e2e_transfer)
    kv.kv_fwd_bwd_host(hv, hx, **kw)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        kv.kv_fwd_bwd_host(hv, hx, **kw)
    secs = time.perf_counter() - t0
    if dist:
        secs = all_reduce_scalar(secs, "max", device=dev)
    mode = args.e2e_transfer
    if mode == "auto":
        mode = "direct" if kv.host_direct_supported() else "staged"
    return {"value": world * n * steps / secs, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * n,
            "d2h_bytes_per_step": 3 * 4 * n, "transfer": mode,
            "host_buffers": "pinned (torch pin_memory)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--bins", type=int, default=32)
    ap.add_argument("--bracket", choices=("mlp", "plain"), default="mlp")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--e2e-transfer", choices=("auto", "staged", "direct"), default="auto",
                    help="how the host-buffer leg moves the data (kv_fwd_bwd_host_ex)")
    ap.add_argument("--pairs", type=int, default=N_PAIRS, help="pairs per GPU (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    rank, local_rank, world = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2108_11560_gb300 import _native as N
    from paper_2108_11560_gb300 import kv

    lib = N.lib()
    n_pairs = args.pairs
    v64, x64 = W.hard_band(n_pairs, seed=1 + 1000 * rank)
    vf = v64.astype(np.float32)
    xf = x64.astype(np.float32)
    vt = torch.from_numpy(vf).to(dev)
    xt = torch.from_numpy(xf).to(dev)
    go = torch.ones(n_pairs, dtype=torch.float32, device=dev)
    outs = {k: torch.empty(n_pairs, dtype=torch.float32, device=dev) for k in ("logk", "dv", "dx")}
    mlp = None
    if args.bracket == "mlp":
        from paper_2108_11560_gb300 import learned
        mlp = learned.default_network(dev)

    def step():
        kv.kv_fwd_bwd_ex(vt, xt, bins=args.bins, bracket=args.bracket, mlp=mlp, grad_out=go,
                         out=outs)

    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = lib.kv_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local_rank) as clocks:
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        # keep the GPU busy (outside the timed region) while the host enqueues the first step, so
        # the first step is not charged with the launch latency of an idle GPU
        torch.cuda._sleep(1 << 21)
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = lib.kv_launch_count() - launches0
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if dist:
        total_ms = all_reduce_scalar(total_ms, "max", device=dev)
    value = world * n_pairs * args.steps / (total_ms / 1e3)

    # end to end: the same call on pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, vf, xf, mlp, dist, dev, world)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peaks, peak_src = _peaks()
    clk = clocks.summary()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 pipe: 128 lanes per SM per clock (an FMA counted as one operation), at the max SM clock
    peak_ops = sms * 128 * sm_mhz * 1e6
    launch_ms = total_ms / args.steps
    # the step's two launches: the fast-path kernel is > 99.8 % of the GPU time (launch list in
    # profiles/launches_bench_hard_band_16M.md), so its launch time is taken as the step time
    if args.bracket == "mlp":
        ops = n_pairs * (FP32_OPS_PER_PAIR + (args.bins + 1) * FP32_OPS_PER_BIN)
        traffic = (n_pairs * TRAFFIC_BYTES_PER_PAIR) if TRAFFIC_BYTES_PER_PAIR else None
        kernel = "kv_mlp_tc_kernel"
    else:  # the plain path is bound by the FP64 bracket; only its FP32 bins are counted
        ops = n_pairs * (args.bins + 1) * FP32_OPS_PER_BIN
        traffic = None
        kernel = "kv_mixed_kernel"
    achieved = ops / (launch_ms / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "Tops/s (FP32 pipe, FMA = 1 op)", "frac": achieved / peak_ops,
                "traffic": traffic, "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz "
                                                      f"({peak_src} max clock)",
                "kernel": kernel}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 bins + extended-precision peak/offset",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if n_pairs == N_PAIRS else f"hard_band_{n_pairs}",
                   "pairs_per_gpu": n_pairs, "bins": args.bins,
                   "bracket": args.bracket, "log_eps": MIXED_LOG_EPS, "io": "float32",
                   "l2": "inputs 134 MB + outputs 201 MB per step, larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "sfu": sfu_utilisation(n_pairs, args.bins, launch_ms, sms, sm_mhz) if args.bracket == "mlp" else None,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(v64.astype(np.float32).astype(np.float64),
                                            x64.astype(np.float32).astype(np.float64), args.bins)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
