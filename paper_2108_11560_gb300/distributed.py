"""Host-side helpers for one process per GPU.

The pairs (v, x) are independent, so the path shards without any exchange: each rank takes a
contiguous share of the arrays and computes it alone.  The only collectives are outside the data
path: the sum of a sharded log-likelihood sum_i log K(v_i, x_i), the maximum of per-rank timings,
and, for training the learned bracket data-parallel, one all-reduce of the network's gradient per
step.  These helpers work with any torch.distributed backend (NCCL on GPUs, gloo in the CPU
tests).
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, local_rank, world_size) from the torchrun environment (0, 0, 1 when absent)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard_bounds(n: int, rank: int, world: int):
    """Contiguous share [lo, hi) of n items for one rank; shares differ in size by at most one
    and cover [0, n) exactly once."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def all_reduce_scalar(value: float, op: str = "sum", device=None) -> float:
    """Sum or maximum of one float over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_collective_device(device))
    dist.all_reduce(t, op={"sum": dist.ReduceOp.SUM, "max": dist.ReduceOp.MAX}[op])
    return float(t.item())


def sharded_loglik(v, x, rank: int, world: int, local_sum, device=None) -> float:
    """sum_i log K(v_i, x_i) over all ranks: each rank passes its share of the full arrays to
    `local_sum` (on a GPU: kv.kv_sum of kv.kv_log) and the partial sums meet in one all-reduce."""
    lo, hi = shard_bounds(len(v), rank, world)
    return all_reduce_scalar(float(local_sum(v[lo:hi], x[lo:hi])), "sum", device)


def _collective_device(device):
    """The device a collective's buffer must live on: the given one, else the current CUDA device
    under the NCCL backend (which takes only CUDA tensors), else the CPU."""
    import torch
    import torch.distributed as dist

    if device is not None:
        return torch.device(device)
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def all_reduce_gradient(loss: float, grad, count: int, device=None):
    """Mean loss and gradient over a batch split across ranks: each rank passes the mean loss and
    gradient over its `count` samples (on a GPU: kv_mlp_loss_grad on its share), and the
    count-weighted sums meet in one all-reduce, so every rank gets the full batch's mean.  This is
    the exchange a data-parallel training step of the learned bracket needs (~4.5k parameters); it
    is a host-side helper, not wired into Mlp.train (training runs on one GPU).  The buffer goes
    to `device`, or by default to the current CUDA device under NCCL and the CPU under gloo.
    Without a process group the arguments come back unchanged.  Returns (loss, grad) with grad
    shaped like the input, in float64."""
    import numpy as np
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(loss), np.asarray(grad, dtype=np.float64)
    g = torch.as_tensor(np.asarray(grad, dtype=np.float64)).reshape(-1)
    buf = torch.cat([g * float(count), torch.tensor([float(loss) * count, float(count)], dtype=torch.float64)])
    buf = buf.to(_collective_device(device))
    dist.all_reduce(buf)
    buf = buf.cpu()
    total = float(buf[-1])
    if total <= 0:
        raise ValueError("no samples on any rank")
    return float(buf[-2]) / total, (buf[:-2] / total).numpy().reshape(np.shape(grad))
