"""Throughput of batched log K_v(x) + d/dv + d/dx (pairs/s) on GB300.

One step = one pass of the whole hot path over the 16,777,216-pair hard-band workload
(75 % v ~ U[0, 50], x log-uniform in [1e-3, 1e3]; 25 % |v - x| < 0.1 v), float32 I/O, mixed path:
bracket (learned MLP with plain fallback), FP32 peak-relative bins, log K, d/dv, d/dx, and the
backward epilogue (the derivatives multiplied by an incoming gradient).  Inputs are resident in
HBM before timing; the working set (134 MB in + 67 MB gradient, 201 MB out) is larger than L2.

After the timed steps (outside the timed region) the outputs of the last timed step are checked
on a seeded sample against the oracle's fixed-bin method in long double at the same bins and eps;
the line carries the errors and the run exits non-zero if any exceeds the accuracy bound.  The
default run also times, each with its own accuracy sample: the learned path at 64 and 128 bins,
the plain FP32 bracket at the headline's bins (the method without the network at its fastest),
the FP64 path at 128 bins on a slice of the same workload, and the other workload configurations
(`configs`: 4096 uniform-small pairs on the FP64 path, the 8M-sample GH log-likelihood through
autograd, 64M learned-bracket evaluation pairs, 128M extreme-range pairs at 64 and 256 bins).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--bins 32]
    python bench.py --path learned|plain|f32|second|f64 [--workload hard_band|uniform_small]
                    [--pairs P] [--no-cpu-baseline] [--no-e2e] [--no-accuracy] [--no-sweep]
    python bench.py --impl reference ...   # the CPU oracle on the host cores (baseline arm)

`--path` selects the timed step (profiling cases): learned = the learned-bracket fast path (the
headline), plain = the mixed path with the FP64 bracket, f32 = Algorithms 1-3 in FP32, second =
the learned path with second derivatives, f64 = the FP64 path (float64 I/O).

Under torchrun each rank runs its own replica of the workload (pairs are independent: weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
F64_LOG_EPS = -52.0 * math.log(2.0)
TOL_MIXED = 2e-6
TOL_F64 = 1e-13
# accuracy samples: the headline step's, and each extra entry's
ACC_SAMPLE = 65_536
ACC_SAMPLE_EXTRA = 16_384
ACC_SAMPLE_F64 = 4_096
ACC_EDGE = 256          # the first and last pairs always belong to the sample
ACC_FALLBACK_MAX = 8_192
F64_SLICE = 1 << 23     # the FP64 path's slice of the workload (134 MB of float64 inputs, larger than L2)

# Algorithmic FP32 work of the learned-bracket fast path, counted operation by operation from
# its formulas with an FMA as one operation and a paired (f32x2) instruction as two:
#   per bin (bins 0..n-1; bin n's terms come from the range check): the abscissa 1, the
#            exponent's x-part (the phi polynomials, or x cosh t from e^{+-s}, which the d/dx
#            integrand shares) 16, the rest of the weight 2, the two derivative integrands 4
#            (+ the tanh polynomial in the warp-blocks that need it, ~3), three sums 3 (plain
#            block sums) or 4.4 (compensated, one Kahan step per eight bins)
#                                                                            -> ~29.6 or ~31 (+ 4 MUFU)
#   per pair: layer 1 and layer 3 on the CUDA cores 256 (layer 2 runs on the tensor cores and
#             is not counted), one peak Newton step, offset constants, endpoint check with bin
#             n's terms, setup and finish ~190                                    -> ~446
# ncu's executed FFMA + FADD + FMUL (+ 2 x FFMA2/FADD2/FMUL2) counters over 4M hard-band pairs (one
# launch of the fast-path kernel each) give these per bin and per pair: for the kernel instance
# with plain block sums (up to PLAIN_SUMS_MAX_BINS bins), from launches at 8 and 32 bins; for the
# instance with compensated block sums (more bins), from launches at 44 and 64 bins.
PLAIN_SUMS_MAX_BINS = 40
FP32_OPS_PER_BIN = 29.606
FP32_OPS_PER_PAIR = 446.32
FP32_OPS_PER_BIN_COMP = 30.986
FP32_OPS_PER_PAIR_COMP = 440.06
MUFU_OPS_PER_BIN = 4
# XU-pipe (MUFU) operations per pair outside the bins from the same captures
# (smsp__inst_executed_pipe_xu x 32: 33.34 per pair and 4.0 per bin), and the XU pipe's lanes
# per SM per clock that ncu's XU percentages are taken against.
MUFU_OPS_PER_PAIR = 33.34
XU_LANES_PER_SM = 32
# Warp instructions issued per pair (smsp__inst_executed x 32 / pairs, same captures): the fast
# path is bound by instruction issue (one warp instruction per SM sub-partition per clock) as
# much as by the FP32 pipe, so the line also reports issue-slot utilisation.
INST_PER_BIN = 26.618
INST_PER_PAIR = 844.6
INST_PER_BIN_COMP = 27.792
INST_PER_PAIR_COMP = 834.3
ISSUE_PER_SM = 4
# DRAM bytes per pair of the fast-path kernel (read + write) from an ncu capture of one full
# 16,777,216-pair launch at 32 bins in steady state (the fourth of five consecutive launches, no
# cache flush between them, so the previous launch's outputs are written back inside it):
# 201.38 MB read + 199.01 MB written.  The algorithmic bytes per pair are v, x, grad_out in and
# log K, d/dv, d/dx out, 4 bytes each (402.65 MB per launch).
TRAFFIC_BYTES_PER_PAIR = (201.376256e6 + 199.007744e6) / 16777216
ALGORITHMIC_BYTES_PER_PAIR = 24
# The counts above hold for the fast-path kernel built from these sources; COUNTS_SOURCE_SHA is
# their hash when the counts were taken.  When the sources change, the line says so and reports
# no traffic until the counters are taken again.
COUNTS_SOURCES = ("kv_mlp.cu", "kv_bins.cuh", "kv_dfloat.cuh")
COUNTS_SOURCE_SHA = "14b10da725e62105"

PATHS = {
    # name: (bracket, second derivatives, float64 I/O)
    "learned": ("mlp", False, False),
    "plain": ("plain", False, False),
    "f32": ("f32", False, False),
    "second": ("mlp", True, False),
    "f64": ("plain", False, True),
}
KERNEL_OF = {"learned": "kv_mlp_tc_kernel", "second": "kv_mlp_tc_kernel", "plain": "kv_mixed_kernel",
             "f32": "kv_plain_f32_kernel", "f64": "kv_f64_kernel"}
WORKLOADS = {"hard_band": (lambda n, seed: W.hard_band(n, seed=seed), N_PAIRS, 1),
             "uniform_small": (lambda n, seed: W.uniform_small(n, seed=seed), 4096, 0)}


def counts_source_sha() -> str:
    h = hashlib.sha256()
    for s in COUNTS_SOURCES:
        with open(os.path.join(ROOT, "paper_2108_11560_gb300", "csrc", s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


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
    ops = n_pairs * (MUFU_OPS_PER_PAIR + bins * MUFU_OPS_PER_BIN)
    achieved = ops / (launch_ms / 1e3)
    peak = sms * XU_LANES_PER_SM * sm_mhz * 1e6
    return {"achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T XU ops/s",
            "frac": achieved / peak,
            "peak_source": f"{sms} SMs x {XU_LANES_PER_SM} XU lanes x {sm_mhz:.0f} MHz (the XU-pipe peak "
                           f"ncu's pipe percentages use)"}


def fp32_ops(bins):
    """FP32 operations per pair of the fast-path kernel instance that runs at this bin count."""
    if bins <= PLAIN_SUMS_MAX_BINS:
        return FP32_OPS_PER_PAIR + bins * FP32_OPS_PER_BIN
    return FP32_OPS_PER_PAIR_COMP + bins * FP32_OPS_PER_BIN_COMP


def issue_utilisation(n_pairs, bins, launch_ms, sms, sm_mhz):
    """Warp instructions issued per second by the fast-path kernel against the SMs' issue rate
    (one warp instruction per sub-partition per clock)."""
    per_pair = (INST_PER_PAIR + bins * INST_PER_BIN if bins <= PLAIN_SUMS_MAX_BINS
                else INST_PER_PAIR_COMP + bins * INST_PER_BIN_COMP)
    achieved = n_pairs * per_pair / 32 / (launch_ms / 1e3)
    peak = sms * ISSUE_PER_SM * sm_mhz * 1e6
    return {"achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T warp instructions/s",
            "frac": achieved / peak, "inst_per_pair": per_pair,
            "peak_source": f"{sms} SMs x {ISSUE_PER_SM} sub-partitions x {sm_mhz:.0f} MHz"}


def fp32_roofline(n_pairs, bins, launch_ms, sms, sm_mhz, peak_src):
    """Algorithmic FP32 operations of the fast-path kernel per launch over its launch time,
    against the FP32 pipe's peak (128 lanes per SM per clock, an FMA counted as one operation)."""
    ops = n_pairs * fp32_ops(bins)
    achieved = ops / (launch_ms / 1e3)
    peak = sms * 128 * sm_mhz * 1e6
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "Tops/s (FP32 pipe, FMA = 1 op)", "frac": achieved / peak,
            "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({peak_src} max clock)"}


def sample_indices(n, k, seed, extra=()):
    """A seeded sample of k indices of [0, n), with the first and last ACC_EDGE indices and the
    given extra ones added."""
    rng = np.random.default_rng(seed)
    parts = [np.arange(min(ACC_EDGE, n)), np.arange(max(n - ACC_EDGE, 0), n),
             rng.choice(n, min(k, n), replace=False)]
    extra = np.asarray(extra, dtype=np.int64)
    if extra.size > ACC_FALLBACK_MAX:
        extra = rng.choice(extra, ACC_FALLBACK_MAX, replace=False)
    parts.append(extra)
    return np.unique(np.concatenate(parts).astype(np.int64))


def accuracy(outs, v64, x64, idx, bins, log_eps, bound, grad_out=None):
    """Maximum errors of the GPU outputs at the sampled indices against the oracle's fixed-bin
    method in long double at the same bins and eps (the errors of Sec. 3.1 taken relative:
    |d log K| / max(1, |log K|); plain relative errors for the derivatives, which must be exactly
    0 at v = 0)."""
    import torch

    import oracle

    it = torch.from_numpy(idx).to(outs["logk"].device)
    g = {k: outs[k].index_select(0, it).double().cpu().numpy() for k in ("logk", "dv", "dx")}
    if grad_out is not None:  # the fused epilogue multiplied the derivatives by grad_out
        go = grad_out.index_select(0, it).double().cpu().numpy()
        g["dv"] = g["dv"] / go
        g["dx"] = g["dx"] / go
    t = time.perf_counter()
    ref = oracle.o1(v64[idx], x64[idx], bins=bins, log_eps=log_eps, precision="long")
    secs = time.perf_counter() - t
    e_l = np.abs(g["logk"] - ref["logk"]) / np.maximum(1.0, np.abs(ref["logk"]))
    z = v64[idx] == 0.0
    e_v = np.where(z, np.where(g["dv"] == 0.0, 0.0, np.inf),
                   np.abs(g["dv"] - ref["dv"]) / np.maximum(np.abs(ref["dv"]), 1e-300))
    e_x = np.abs(g["dx"] - ref["dx"]) / np.maximum(np.abs(ref["dx"]), 1e-300)
    worst = max(float(e_l.max()), float(e_v.max()), float(e_x.max()))
    return {"max_rel_logk": float(e_l.max()), "max_rel_dv": float(e_v.max()),
            "max_rel_dx": float(e_x.max()),
            "max_abs_logk": float(np.abs(g["logk"] - ref["logk"]).max()),  # = relative error of K
            "pairs": int(idx.size), "bound": bound,
            "ok": bool(worst <= bound),
            "reference": f"oracle O1 in long double, {bins} bins, log eps {log_eps:.4g}",
            "oracle_s": round(secs, 2)}


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
    kw = dict(bins=args.bins, bracket="mlp", mlp=mlp, out=hout, transfer=args.e2e_transfer)
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


def timed_steps(step, steps, warmup, stream):
    """CUDA-event times (ms) of `steps` calls of step() after `warmup` untimed ones."""
    import torch

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda._sleep(1 << 21)  # the GPU is busy while the host enqueues the first timed step
    ev[0].record(stream)
    for k in range(steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[-1]), [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]


def fallback_pairs(kv, vt, xt, kw):
    """Indices of the pairs that fell back to the plain bracket (status bit) and the rate, from
    one more untimed call with the same arguments (the results are deterministic)."""
    import torch

    from paper_2108_11560_gb300 import _native as N

    s = kv.kv_fwd_bwd_ex(vt, xt, status=True, **kw)["status"]
    fb = torch.nonzero((s & N.KV_PAIR_FALLBACK) != 0).flatten().cpu().numpy()
    return fb, fb.size / max(vt.numel(), 1)


def extra_entries(args, kv, mlp, vf, xf, v64c, x64c, dev, stream, sms, sm_mhz, peak_src, check):
    """The sweep of the learned path over 64 and 128 bins, the plain FP32 bracket at the headline's
    bins and the FP64 path at 128 bins on a slice, each timed with CUDA events and each with its
    own accuracy sample."""
    import torch

    n = vf.size
    vt = torch.from_numpy(vf).to(dev)
    xt = torch.from_numpy(xf).to(dev)
    out = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in ("logk", "dv", "dx")}
    res = {"sweep": {}, "f32_bracket": None, "fp64_plain": None}
    runs = [("mlp", b) for b in (64, 128) if b != args.bins] + [("f32", args.bins)]
    for bracket, bins in runs:
        kw = dict(bins=bins, bracket=bracket, mlp=mlp if bracket == "mlp" else None)
        total, _ = timed_steps(lambda: kv.kv_fwd_bwd_ex(vt, xt, out=out, **kw), args.steps, args.warmup, stream)
        ms = total / args.steps
        e = {"bins": bins, "value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "pairs": n}
        if bracket == "mlp":
            e["frac_fp32"] = fp32_roofline(n, bins, ms, sms, sm_mhz, peak_src)["frac"]
        if check:
            fb, rate = fallback_pairs(kv, vt, xt, kw)
            e["fallback_rate"] = rate
            idx = sample_indices(n, ACC_SAMPLE_EXTRA, 1000 + bins, fb)
            e["accuracy"] = accuracy(out, v64c, x64c, idx, bins, MIXED_LOG_EPS, TOL_MIXED)
        if bracket == "mlp":
            res["sweep"][str(bins)] = e
        else:
            e["kernel"] = KERNEL_OF["f32"]
            res["f32_bracket"] = e
    del vt, xt, out
    # the FP64 path on the first F64_SLICE pairs (the float32-cast inputs in double)
    m = min(F64_SLICE, n)
    v64t = torch.from_numpy(v64c[:m].copy()).to(dev)
    x64t = torch.from_numpy(x64c[:m].copy()).to(dev)
    o64 = {k: torch.empty(m, dtype=torch.float64, device=dev) for k in ("logk", "dv", "dx")}
    total, _ = timed_steps(lambda: kv.kv_fwd_bwd_ex(v64t, x64t, bins=128, out=o64), max(2, args.steps // 3),
                           args.warmup, stream)
    ms = total / max(2, args.steps // 3)
    e = {"bins": 128, "value": m / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "pairs": m,
         "slice": f"first {m} pairs of the workload, float64 I/O", "kernel": KERNEL_OF["f64"]}
    if check:
        idx = sample_indices(m, ACC_SAMPLE_F64, 2000)
        e["accuracy"] = accuracy(o64, v64c[:m], x64c[:m], idx, 128, F64_LOG_EPS, TOL_F64)
    res["fp64_plain"] = e
    return res


def vectorised_scaling(args, kv, mlp, dev, stream):
    """Sec. 3.4's vectorised timing: one call on arrays of N = 10 ... 10^8 pairs of the paper's
    inputs (v = 10^{2r} - 1, x = 10^{3r - 1}), at the library's default bins.  Per N: the device
    time of a call (CUDA events, calls back to back) and the wall time of one blocking call from
    the host (launch + synchronize; what a user waits for on small arrays), for the learned path
    and, up to 10^6 pairs, the FP64 path."""
    import torch

    res = {"inputs": "v = 10^(2r) - 1, x = 10^(3r - 1), r ~ U[0, 1] per element (seed 8)",
           "learned": {}, "fp64": {}}
    reps = max(5, args.steps)
    for e in range(1, 9):
        n = 10 ** e
        v, x = W.paper_scaling(n, seed=8)
        for path, dt, limit in (("learned", torch.float32, 10 ** 8), ("fp64", torch.float64, 10 ** 6)):
            if n > limit:
                continue
            vt = torch.tensor(v, dtype=dt, device=dev)
            xt = torch.tensor(x, dtype=dt, device=dev)
            kw = dict(bracket="mlp", mlp=mlp) if path == "learned" else dict(bins=128)
            out = kv.kv_fwd_bwd_ex(vt, xt, **kw)
            total, _ = timed_steps(lambda: kv.kv_fwd_bwd_ex(vt, xt, out=out, **kw), reps, 3, stream)
            wall = []
            for _ in range(reps):
                t = time.perf_counter()
                kv.kv_fwd_bwd_ex(vt, xt, out=out, **kw)
                torch.cuda.synchronize()
                wall.append((time.perf_counter() - t) * 1e3)
            res[path][str(n)] = {"device_ms": total / reps, "wall_ms": statistics.median(wall)}
            del vt, xt, out
    return res


def config_entries(args, kv, mlp, dev, stream, check):
    """The other workload configurations, each timed with CUDA events and checked on a sample:
    uniform_small (4096 pairs, FP64, 128 bins, log K only), the GH log-likelihood through
    autograd (8M float32 samples, forward with fused derivatives, deterministic sum, backward
    epilogue), the learned-bracket evaluation (64M fresh pairs, network trained on 1M plain
    brackets of the same distribution) and the extreme range (128M pairs at 64 and 256 bins, its
    own network, against the FP64 path on a 2M slice)."""
    import torch

    from paper_2108_11560_gb300 import learned

    res = {}
    reps = max(3, args.steps // 2)
    # uniform_small: 4096 pairs, FP64, log K only (kv_log)
    v, x = W.uniform_small(4096, seed=0)
    vt, xt = torch.from_numpy(v).to(dev), torch.from_numpy(x).to(dev)
    out = torch.empty_like(vt)
    total, _ = timed_steps(lambda: kv.kv_fwd_bwd_ex(vt, xt, bins=128, want=("logk",), out={"logk": out}),
                           reps * 4, args.warmup, stream)
    ms = total / (reps * 4)
    e = {"pairs": 4096, "bins": 128, "value": 4096 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
         "path": "FP64, log K only"}
    if check:
        import oracle
        ref = oracle.o1(v, x, bins=128, precision="long")["logk"]
        g = out.double().cpu().numpy()
        e["accuracy"] = {"max_rel_logk": float((np.abs(g - ref) / np.maximum(1.0, np.abs(ref))).max()),
                         "pairs": 4096, "bound": TOL_F64}
        e["accuracy"]["ok"] = e["accuracy"]["max_rel_logk"] <= TOL_F64
    res["uniform_small_4096"] = e
    # GH log-likelihood through autograd
    n = 8_388_608
    lam, xg, *_ = W.gh_likelihood(n, seed=2)
    lt = torch.from_numpy(lam).to(dev).requires_grad_(True)
    xt = torch.from_numpy(xg).to(dev).requires_grad_(True)
    loss = [None]

    def gh_step():
        lt.grad = None
        xt.grad = None
        lk = kv.log_besselk(lt, xt, bins=40, bracket="mlp", mlp=mlp)
        loss[0] = kv.kv_sum(lk.detach())
        lk.backward(torch.ones_like(lk))
    total, _ = timed_steps(gh_step, reps, args.warmup, stream)
    ms = total / reps
    e = {"pairs": n, "bins": 40, "value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
         "path": "learned bracket through torch.autograd: forward with fused derivatives, "
                 "deterministic sum, backward epilogue"}
    if check:
        idx = sample_indices(n, ACC_SAMPLE_F64, 3000)
        outs = {"logk": kv.log_besselk(lt.detach(), xt.detach(), bins=40, bracket="mlp", mlp=mlp),
                "dv": lt.grad, "dx": xt.grad}
        e["accuracy"] = accuracy(outs, lam.astype(np.float64), xg.astype(np.float64), idx, 40,
                                 MIXED_LOG_EPS, TOL_MIXED)
        e["loglik"] = float(loss[0].item())
    res["gh_likelihood_8M"] = e
    del lt, xt
    # learned-bracket evaluation: 64M fresh pairs, a network trained on 1M plain brackets
    net4, _ = learned.train_network(dev, domain="uniform")
    n = 64 * 1024 * 1024
    v, x = W.learned_bracket(n, seed=6)
    vf, xf = v.astype(np.float32), x.astype(np.float32)
    del v, x
    vt, xt = torch.from_numpy(vf).to(dev), torch.from_numpy(xf).to(dev)
    o = kv.kv_fwd_bwd_ex(vt, xt, bins=40, bracket="mlp", mlp=net4)
    total, _ = timed_steps(lambda: kv.kv_fwd_bwd_ex(vt, xt, bins=40, bracket="mlp", mlp=net4, out=o), reps,
                           args.warmup, stream)
    ms = total / reps
    e = {"pairs": n, "bins": 40, "value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
         "network": "trained on 1M plain brackets, v ~ U[0, 200], x log-uniform in [1e-4, 1e4]"}
    if check:
        fb, rate = fallback_pairs(kv, vt, xt, dict(bins=40, bracket="mlp", mlp=net4))
        e["fallback_rate"] = rate
        idx = sample_indices(n, ACC_SAMPLE_F64, 4000, fb)
        e["accuracy"] = accuracy(o, vf.astype(np.float64), xf.astype(np.float64), idx, 40, MIXED_LOG_EPS,
                                 TOL_MIXED)
    res["learned_bracket_eval_64M"] = e
    del vt, xt, o, vf, xf
    # extreme range: 128M pairs, its own network; the FP64 path on a 2M slice
    net5, _ = learned.train_network(dev, domain="extreme", seed=4)
    n = 128 * 1024 * 1024
    v, x = W.extreme_range(n, seed=5)
    vf, xf = v.astype(np.float32), x.astype(np.float32)
    del v, x
    vt, xt = torch.from_numpy(vf).to(dev), torch.from_numpy(xf).to(dev)
    m = 1 << 21
    v64, x64 = vf[:m].astype(np.float64), xf[:m].astype(np.float64)
    v64t, x64t = torch.from_numpy(v64).to(dev), torch.from_numpy(x64).to(dev)
    for bins in (64, 256):
        o = kv.kv_fwd_bwd_ex(vt, xt, bins=bins, bracket="mlp", mlp=net5)
        total, _ = timed_steps(lambda: kv.kv_fwd_bwd_ex(vt, xt, bins=bins, bracket="mlp", mlp=net5, out=o),
                               max(2, reps // 2), args.warmup, stream)
        ms = total / max(2, reps // 2)
        o64 = kv.kv_fwd_bwd_ex(v64t, x64t, bins=bins)
        t64, _ = timed_steps(lambda: kv.kv_fwd_bwd_ex(v64t, x64t, bins=bins, out=o64), 2, 3, stream)
        e = {"pairs": n, "bins": bins, "value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
             "network": "trained on 1M plain brackets of the extreme range",
             "fp64_plain": {"pairs": m, "value": m / (t64 / 2 / 1e3), "unit": UNIT,
                            "slice": f"first {m} pairs, float64 I/O"}}
        if check:
            fb, rate = fallback_pairs(kv, vt, xt, dict(bins=bins, bracket="mlp", mlp=net5))
            e["fallback_rate"] = rate
            idx = sample_indices(n, ACC_SAMPLE_F64, 5000 + bins, fb)
            e["accuracy"] = accuracy(o, vf.astype(np.float64), xf.astype(np.float64), idx, bins,
                                     MIXED_LOG_EPS, TOL_MIXED)
            k = sample_indices(m, 1024, 6000 + bins)
            e["fp64_plain"]["accuracy"] = accuracy(o64, v64, x64, k, bins, F64_LOG_EPS, TOL_F64)
        res[f"extreme_range_128M_{bins}"] = e
        del o, o64
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--bins", type=int, default=0, help="0: 32 (128 on the FP64 path)")
    ap.add_argument("--path", choices=tuple(PATHS), default="learned")
    ap.add_argument("--bracket", choices=("mlp", "plain", "f32"), default=None,
                    help="the same as --path learned|plain|f32")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="hard_band")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the accuracy samples (profiling runs)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the extra timed entries (profiling runs)")
    ap.add_argument("--e2e-transfer", choices=("auto", "staged", "direct"), default="auto",
                    help="how the host-buffer leg moves the data (kv_fwd_bwd_host_ex)")
    ap.add_argument("--pairs", type=int, default=0, help="pairs per GPU (0: the workload's size)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.bracket is not None:
        args.path = {"mlp": "learned", "plain": "plain", "f32": "f32"}[args.bracket]
    bracket, second, f64io = PATHS[args.path]
    if args.bins == 0:
        args.bins = 128 if f64io else 32
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
    gen, default_n, seed = WORKLOADS[args.workload]
    n_pairs = args.pairs or default_n
    headline = args.path == "learned" and args.workload == "hard_band"
    v64, x64 = gen(n_pairs, seed + 1000 * rank)
    io = np.float64 if f64io else np.float32
    vf = v64.astype(io)
    xf = x64.astype(io)
    # the inputs the GPU sees, in double, for the oracle
    v64c = vf.astype(np.float64)
    x64c = xf.astype(np.float64)
    tdt = torch.float64 if f64io else torch.float32
    vt = torch.from_numpy(vf).to(dev)
    xt = torch.from_numpy(xf).to(dev)
    go = torch.ones(n_pairs, dtype=tdt, device=dev)
    outs = {k: torch.empty(n_pairs, dtype=tdt, device=dev) for k in ("logk", "dv", "dx")}
    if second:
        outs.update({k: torch.empty(n_pairs, dtype=tdt, device=dev) for k in ("d2v", "dvx", "d2x")})
    mlp = None
    if bracket == "mlp":
        from paper_2108_11560_gb300 import learned
        mlp = learned.default_network(dev)
    kw = dict(bins=args.bins, bracket=bracket, mlp=mlp, second=second)

    def step():
        kv.kv_fwd_bwd_ex(vt, xt, grad_out=None if second else go, out=outs, **kw)

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
    if headline and not args.no_e2e:
        e2e = end_to_end(args, vf, xf, mlp, dist, dev, world)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peaks, peak_src = _peaks()
    clk = clocks.summary()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    launch_ms = total_ms / args.steps
    check = not args.no_accuracy
    acc = None
    fb_rate = None
    if check:
        # the last timed step's outputs, on a seeded sample with the fallback pairs added
        fb = np.zeros(0, dtype=np.int64)
        if bracket == "mlp":
            fb, fb_rate = fallback_pairs(kv, vt, xt, kw)
        idx = sample_indices(n_pairs, ACC_SAMPLE, 7, fb)
        acc = accuracy(outs, v64c, x64c, idx, args.bins, F64_LOG_EPS if f64io else MIXED_LOG_EPS,
                       TOL_F64 if f64io else TOL_MIXED, grad_out=None if second else go)
        acc["fallback_rate"] = fb_rate
    sha = counts_source_sha()
    counts_current = sha == COUNTS_SOURCE_SHA
    roofline = None
    sfu = None
    issue = None
    if bracket == "mlp" and not second:
        # the step's two launches: the fast-path kernel is > 99.8 % of the GPU time (ncu launch
        # list of this command), so its launch time is taken as the step time
        roofline = fp32_roofline(n_pairs, args.bins, launch_ms, sms, sm_mhz, peak_src)
        roofline["traffic"] = (n_pairs * TRAFFIC_BYTES_PER_PAIR
                               if (TRAFFIC_BYTES_PER_PAIR and counts_current) else None)
        roofline["algorithmic_bytes"] = n_pairs * ALGORITHMIC_BYTES_PER_PAIR
        roofline["kernel"] = KERNEL_OF[args.path]
        roofline["counts_source_sha"] = sha
        roofline["counts_current"] = counts_current
        sfu = sfu_utilisation(n_pairs, args.bins, launch_ms, sms, sm_mhz)
        sfu["counts_current"] = counts_current
        issue = issue_utilisation(n_pairs, args.bins, launch_ms, sms, sm_mhz)
        issue["counts_current"] = counts_current
    io_desc = "float64" if f64io else "float32"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if f64io else "f32 bins + extended-precision peak/offset",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if headline and n_pairs == N_PAIRS else f"{args.workload}_{n_pairs}",
                   "pairs_per_gpu": n_pairs, "bins": args.bins, "path": args.path,
                   "bracket": bracket, "second_derivatives": second,
                   "log_eps": F64_LOG_EPS if f64io else MIXED_LOG_EPS, "io": io_desc,
                   "l2": "inputs 134 MB + outputs 201 MB per step, larger than L2 (no flush)"
                         if n_pairs >= N_PAIRS else "profiling case",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "sfu": sfu,
        "issue": issue,
        "accuracy": acc,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
    }
    if headline and not args.no_sweep:
        line.update(extra_entries(args, kv, mlp, vf, xf, v64c, x64c, dev, stream, sms, sm_mhz,
                                  peak_src, check))
        if line["f32_bracket"]:
            line["learned_vs_f32_bracket"] = value / world / line["f32_bracket"]["value"]
        if line["fp64_plain"]:
            line["learned_vs_fp64_plain"] = value / world / line["fp64_plain"]["value"]
        line["configs"] = config_entries(args, kv, mlp, dev, stream, check)
        line["vectorised_scaling"] = vectorised_scaling(args, kv, mlp, dev, stream)
    if world == 1 and not args.no_cpu_baseline and not f64io:
        line["cpu_baseline"] = cpu_baseline(v64c, x64c, args.bins)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    oks = [line["accuracy"]] + [e.get("accuracy") for e in line.get("sweep", {}).values()]
    oks += [(line.get(k) or {}).get("accuracy") for k in ("f32_bracket", "fp64_plain")]
    for e in (line.get("configs") or {}).values():
        oks += [e.get("accuracy"), (e.get("fp64_plain") or {}).get("accuracy")]
    if any(a is not None and not a["ok"] for a in oks):
        print("accuracy bound exceeded", file=sys.stderr)
        return 3
    return 0


if __name__ == "__main__":
    sys.exit(main())
