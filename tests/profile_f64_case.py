"""Small FP64-path case for profiling (run by hand under ncu, not collected by pytest):
1,048,576 uniform-small pairs (v ~ U[0, 10], x log-uniform in [1e-2, 1e2]), 128 bins, one
fused launch of kv_fwd_bwd."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_2108_11560_gb300 import kv  # noqa: E402
from paper_2108_11560_gb300 import workloads as W  # noqa: E402

if __name__ == "__main__":
    v, x = W.uniform_small(1 << 20, seed=0)
    dev = torch.device("cuda", 0)
    vt = torch.tensor(v, device=dev)
    xt = torch.tensor(x, device=dev)
    lk, dv, dx = kv.kv_fwd_bwd(vt, xt, bins=128)
    torch.cuda.synchronize()
    print("ok", float(lk.sum()), float(dv.sum()), float(dx.sum()))
