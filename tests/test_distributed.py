"""Multi-process host logic on CPU (gloo, world size 2): shards cover the pairs exactly once, the
sharded log-likelihood equals the serial one, and the data-parallel gradient of the learned
bracket equals the full batch's.  The per-rank partial sums and gradients come from the CPU
oracles here (the GPU path computes them with kv_sum and kv_mlp_loss_grad on each rank's
device)."""
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


def _grad_batch():
    from oracle import mlp as omlp
    from paper_2108_11560_gb300 import workloads as W

    rng = np.random.default_rng(17)
    p = rng.standard_normal(omlp.NPARAMS) * 0.1
    v, x = W.learned_bracket(301, seed=18)
    tp = omlp.peak(v, x)
    t0 = np.maximum(tp - rng.uniform(0.01, 2.0, v.size), 0.0)
    t1 = tp + rng.uniform(0.01, 4.0, v.size)
    return p, v, x, t0, tp, t1


def _grad_worker(rank, world, port, out):
    import torch.distributed as dist

    from oracle import mlp as omlp

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, v, x, t0, tp, t1 = _grad_batch()
        lo, hi = D.shard_bounds(v.size, rank, world)  # unequal shares: 151 and 150 samples
        loss, g = omlp.loss_grad(p, v[lo:hi], x[lo:hi], t0[lo:hi], tp[lo:hi], t1[lo:hi])
        # the collective's buffer goes to the CPU under gloo (to the current GPU under NCCL)
        assert D._collective_device(None).type == "cpu"
        out[rank] = D.all_reduce_gradient(loss, g, hi - lo)
    finally:
        dist.destroy_process_group()


def test_data_parallel_gradient_gloo_world_2():
    from oracle import mlp as omlp

    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_grad_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    p, v, x, t0, tp, t1 = _grad_batch()
    loss, g = omlp.loss_grad(p, v, x, t0, tp, t1)
    for r in range(world):
        lr, gr = out[r]
        assert abs(lr - loss) <= 1e-12 * abs(loss)
        assert np.allclose(gr, g, rtol=1e-12, atol=1e-15 * np.abs(g).max())
    # without a process group the arguments come back unchanged
    l1, g1 = D.all_reduce_gradient(loss, g, v.size)
    assert l1 == loss and np.array_equal(g1, g)
