"""Small cases of the learned path with second derivatives and of the FP32-bracket path, for
profiling (run by hand under ncu, not collected by pytest): 4,194,304 hard-band pairs in float32,
32 bins, one warm-up call then one profiled call of kv_fwd_bwd_ex.

    python tests/profile_paths_case.py second     # learned bracket + second derivatives
    python tests/profile_paths_case.py f32        # Algorithms 1-3 in FP32 (first derivatives)
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2108_11560_gb300 import kv, learned  # noqa: E402
from paper_2108_11560_gb300 import workloads as W  # noqa: E402

if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "second"
    dev = torch.device("cuda", 0)
    v, x = W.hard_band(1 << 22, seed=1)
    vt = torch.tensor(v, dtype=torch.float32, device=dev)
    xt = torch.tensor(x, dtype=torch.float32, device=dev)
    if which == "second":
        kw = dict(bins=32, bracket="mlp", mlp=learned.default_network(dev), second=True)
    elif which == "f32":
        kw = dict(bins=32, bracket="f32")
    else:
        raise SystemExit("usage: profile_paths_case.py [second|f32]")
    out = kv.kv_fwd_bwd_ex(vt, xt, **kw)
    out = kv.kv_fwd_bwd_ex(vt, xt, out=out, **kw)
    torch.cuda.synchronize()
    print("ok", which, float(out["logk"].double().sum()))
