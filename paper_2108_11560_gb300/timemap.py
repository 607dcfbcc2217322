"""Per-(v, x) time maps (Sec. 3.2): the time per pair of each path for batches that hold one
(v, x) point each, over a grid of the paper's evaluation domain (v in [0, 99], x in
[10^-1, 10^2.1], the grid of Sec. 3 thinned), so that regions where a path slows down show.

The paper measured that its integration method takes about the same time everywhere while the
series, continued-fraction and asymptotic methods do not; on the GPU every pair of a warp runs
the same fixed trip counts, so the map is flat up to the data-dependent parts (FindRange's
doublings, the learned range's Newton corrections and fallbacks).

    python -m paper_2108_11560_gb300.timemap [--pairs 1048576] [--nv 9] [--nx 9]
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import kv, learned

PATHS = {
    "fp64": dict(dtype=torch.float64, bins=128, bracket="plain"),
    "mixed_fp64_bracket": dict(dtype=torch.float32, bins=32, bracket="plain"),
    "f32": dict(dtype=torch.float32, bins=32, bracket="f32"),
    "learned": dict(dtype=torch.float32, bins=32, bracket="mlp"),
}


def grid(nv: int, nx: int):
    """The paper's evaluation grid (v = 10^(i/40) - 1 for i = 0..80, x = 10^(i/40) for
    i = -40..84), thinned to nv x nx points with both ends kept."""
    iv = np.unique(np.round(np.linspace(0, 80, nv)).astype(int))
    ix = np.unique(np.round(np.linspace(-40, 84, nx)).astype(int))
    return 10.0 ** (iv / 40.0) - 1.0, 10.0 ** (ix / 40.0)


def time_map(paths=("fp64", "learned"), pairs: int = 1 << 20, nv: int = 9, nx: int = 9, reps: int = 3,
             device=None, mlp=None):
    """{path: (v values, x values, ns per pair [nv, nx])} with CUDA-event timing of `reps` calls
    per point after one warm-up call."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    vs, xs = grid(nv, nx)
    if "learned" in paths and mlp is None:
        mlp = learned.default_network(device)
    out = {}
    for name in paths:
        cfg = PATHS[name]
        n = pairs if name != "fp64" and name != "mixed_fp64_bracket" else max(pairs // 16, 1024)
        t = np.empty((vs.size, xs.size))
        v = torch.empty(n, dtype=cfg["dtype"], device=device)
        x = torch.empty(n, dtype=cfg["dtype"], device=device)
        for a, vv in enumerate(vs):
            for b, xx in enumerate(xs):
                v.fill_(float(vv))
                x.fill_(float(xx))
                kw = dict(bins=cfg["bins"], bracket=cfg["bracket"], mlp=mlp if cfg["bracket"] == "mlp" else None)
                res = kv.kv_fwd_bwd_ex(v, x, **kw)
                torch.cuda.synchronize(device)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    kv.kv_fwd_bwd_ex(v, x, out=res, **kw)
                e1.record()
                torch.cuda.synchronize(device)
                t[a, b] = e0.elapsed_time(e1) * 1e6 / (reps * n)
        out[name] = (vs, xs, t)
    return out


def format_map(vs, xs, t) -> str:
    head = "v \\ x    " + " ".join(f"{x:8.3g}" for x in xs)
    rows = [f"{v:8.3g} " + " ".join(f"{c:8.3f}" for c in row) for v, row in zip(vs, t)]
    return "\n".join([head] + rows)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--pairs", type=int, default=1 << 20)
    ap.add_argument("--nv", type=int, default=9)
    ap.add_argument("--nx", type=int, default=9)
    ap.add_argument("--paths", default="fp64,mixed_fp64_bracket,f32,learned")
    args = ap.parse_args()
    maps = time_map(tuple(args.paths.split(",")), args.pairs, args.nv, args.nx)
    for name, (vs, xs, t) in maps.items():
        print(f"\n[{name}] ns per pair (max/min {t.max() / t.min():.2f})")
        print(format_map(vs, xs, t))


if __name__ == "__main__":
    main()
