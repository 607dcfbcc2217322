"""The learned bracket: a handle on the library's 2-64-64-2 MLP, its training driver and the
default network used by the fast path.

Everything here is argument marshalling around the C ABI (kv_mlp_*); the forward pass,
backward pass and Adam update run in the library's CUDA kernels.  Training data: pairs drawn
from the learned-bracket workload (v ~ U[0, 200], x log-uniform in [1e-4, 1e4]) with targets from
the plain FP64 bracket (kv_bracket, Algorithms 1-3) at a range eps of e^-26, six nats wider than
the mixed path's e^-20, so that predictions land inside the check window
[log eps - 12, log eps] of the fast path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import _native as N
from . import kv
from . import workloads as W

#: range eps of the training targets (the mixed path uses e^-20; the check accepts e^-32..e^-20)
TRAIN_LOG_EPS = -26.0
#: default training schedule: (Adam steps, learning rate) stages
SCHEDULE = ((6000, 2e-3), (4000, 5e-4), (3000, 1.25e-4), (2000, 3e-5))
BATCH = 8192
TRAIN_PAIRS = 1 << 20


class Mlp:
    """An owned kv_mlp handle (device memory freed with the object)."""

    def __init__(self, handle: int):
        self.handle = handle

    @classmethod
    def create(cls, seed: int = 0) -> "Mlp":
        h = ctypes.c_void_p()
        N.check(N.lib().kv_mlp_create(seed, ctypes.byref(h)), "kv_mlp_create")
        return cls(h.value)

    @classmethod
    def load(cls, path: str) -> "Mlp":
        h = ctypes.c_void_p()
        N.check(N.lib().kv_mlp_load(path.encode(), ctypes.byref(h)), "kv_mlp_load")
        return cls(h.value)

    def save(self, path: str) -> None:
        N.check(N.lib().kv_mlp_save(self.handle, path.encode()), "kv_mlp_save")

    def free(self) -> None:
        if self.handle:
            N.lib().kv_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(N.KV_MLP_NPARAMS, dtype=np.float32)
        N.check(N.lib().kv_mlp_get_params(self.handle, out.ctypes.data, out.size), "kv_mlp_get_params")
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        N.check(N.lib().kv_mlp_set_params(self.handle, p.ctypes.data, p.size), "kv_mlp_set_params")

    def train(self, v, x, t0, t1, steps: int, batch: int = BATCH, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, seed: int = 0):
        """Adam steps on float64 CUDA tensors; returns the per-step mean losses (float32)."""
        for t in (v, x, t0, t1):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("training tensors must be contiguous float64 CUDA tensors")
        losses = torch.empty(max(steps, 1), dtype=torch.float32, device=v.device)
        a = N.KvTrainArgs()
        a.v, a.x, a.t0, a.t1 = v.data_ptr(), x.data_ptr(), t0.data_ptr(), t1.data_ptr()
        a.n = v.numel()
        a.batch, a.steps = batch, steps
        a.lr, a.beta1, a.beta2, a.adam_eps = lr, beta1, beta2, eps
        a.seed = seed
        a.loss_out = losses.data_ptr()
        a.stream = torch.cuda.current_stream(v.device).cuda_stream
        N.check(N.lib().kv_mlp_train(self.handle, ctypes.byref(a)), "kv_mlp_train")
        return losses[:steps].cpu().numpy()

    def loss_grad(self, v, x, t0, t1):
        """(mean loss, gradient) of one batch (all of v), without an update."""
        loss = torch.empty((), dtype=torch.float64, device=v.device)
        grads = torch.empty(N.KV_MLP_NPARAMS, dtype=torch.float32, device=v.device)
        P = lambda t: ctypes.c_void_p(t.data_ptr())
        N.check(N.lib().kv_mlp_loss_grad(self.handle, P(v), P(x), P(t0), P(t1), v.numel(), P(loss),
                                         P(grads), torch.cuda.current_stream(v.device).cuda_stream),
                "kv_mlp_loss_grad")
        return loss.item(), grads.cpu().numpy()

    def predict(self, v, x):
        """Raw (t0, t1) predictions on float32 CUDA tensors."""
        t0 = torch.empty_like(v)
        t1 = torch.empty_like(v)
        P = lambda t: ctypes.c_void_p(t.data_ptr())
        N.check(N.lib().kv_mlp_predict(self.handle, P(v), P(x), P(t0), P(t1), v.numel(), N.KV_MIXED,
                                       torch.cuda.current_stream(v.device).cuda_stream),
                "kv_mlp_predict")
        return t0, t1


#: training distributions: "uniform" is v ~ U[0, 200] (the 1M-pair learned-bracket recipe);
#: "mixed" (the default network's) puts half of the orders log-uniform in [1e-3, 200]
DOMAINS = {"uniform": W.learned_bracket, "mixed": W.learned_bracket_mixed,
           "extreme": W.extreme_training}


def training_set(device, n: int = TRAIN_PAIRS, seed: int = 3, log_eps: float = TRAIN_LOG_EPS,
                 domain: str = "mixed"):
    """(v, x, t0, t1) float64 CUDA tensors: learned-bracket inputs cast through float32 (what the
    fast path sees) with targets from the plain FP64 bracket."""
    v, x = DOMAINS[domain](n, seed=seed)
    v = torch.tensor(v.astype(np.float32), dtype=torch.float64, device=device)
    x = torch.tensor(x.astype(np.float32), dtype=torch.float64, device=device)
    t0, _, t1, _ = kv.kv_bracket(v, x, log_eps=log_eps)
    return v, x, t0, t1


def train_network(device, n: int = TRAIN_PAIRS, seed: int = 3, schedule=SCHEDULE,
                  batch: int = BATCH, init_seed: int = 1, domain: str = "mixed"):
    """A freshly trained network (and its loss curve)."""
    v, x, t0, t1 = training_set(device, n, seed, domain=domain)
    net = Mlp.create(init_seed)
    losses = []
    for k, (steps, lr) in enumerate(schedule):
        losses.append(net.train(v, x, t0, t1, steps=steps, batch=batch, lr=lr, seed=seed + 17 * k))
    return net, np.concatenate(losses)


_DEFAULT = {}
_LOCK = threading.Lock()
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "mlp_default.kvmlp")


def default_network(device=None) -> Mlp:
    """The network the fast path uses by default: loaded from the in-tree cache file if present,
    otherwise trained on this GPU (a few seconds) and cached."""
    device = torch.device(device or "cuda")
    idx = device.index if device.index is not None else torch.cuda.current_device()
    with _LOCK:
        if idx not in _DEFAULT:
            with torch.cuda.device(idx):
                net = None
                if os.path.exists(_CACHE):
                    try:
                        net = Mlp.load(_CACHE)
                    except N.KvError:
                        net = None
                if net is None:
                    net, _ = train_network(torch.device("cuda", idx))
                    torch.cuda.synchronize(idx)
                    try:
                        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
                        net.save(_CACHE)
                    except (N.KvError, OSError):
                        pass
                _DEFAULT[idx] = net
        return _DEFAULT[idx]
