"""Multi-process host logic on CPU (gloo, world size 2): shards cover the pairs exactly once and
the sharded log-likelihood equals the serial one.  The per-rank partial sums come from the CPU
oracle here (the GPU path computes them with kv_sum on each rank's device)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2108_11560_gb300 import distributed as D


def test_shard_bounds_cover_exactly_once():
    for n in (0, 1, 7, 1000, 16_777_216 + 3):
        for world in (1, 2, 3, 8):
            seen = 0
            prev = 0
            sizes = []
            for r in range(world):
                lo, hi = D.shard_bounds(n, r, world)
                assert lo == prev and hi >= lo
                prev = hi
                seen += hi - lo
                sizes.append(hi - lo)
            assert prev == n and seen == n
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard_bounds(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    from paper_2108_11560_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lam, x, *_ = W.gh_likelihood(5001, seed=2)
        local = lambda a, b: oracle.o1(a.astype(np.float64), b.astype(np.float64), bins=32,
                                       log_eps=-20.0, threads=1)["logk"].sum()
        total = D.sharded_loglik(lam, x, rank, world, local)
        tmax = D.all_reduce_scalar(float(rank + 1), "max")
        out[rank] = (total, tmax)
    finally:
        dist.destroy_process_group()


def test_sharded_loglik_gloo_world_2():
    import oracle
    from paper_2108_11560_gb300 import workloads as W

    oracle.build()
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    lam, x, *_ = W.gh_likelihood(5001, seed=2)
    serial = oracle.o1(lam.astype(np.float64), x.astype(np.float64), bins=32, log_eps=-20.0)["logk"].sum()
    for r in range(world):
        total, tmax = out[r]
        assert abs(total - serial) <= 1e-9 * abs(serial)
        assert tmax == float(world)
