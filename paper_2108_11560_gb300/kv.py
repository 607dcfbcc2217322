"""PyTorch binding of the C ABI (include/kv.h): argument marshalling only.

Every function here takes CUDA tensors, passes their device pointers and the current CUDA
stream to libkv.so and returns tensors it allocated with PyTorch.  There is no CPU path: CPU
tensors, or a missing library, raise.  float64 inputs select the FP64 path (KV_F64), float32
inputs the mixed path (KV_MIXED).
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return N.KV_F64
    if t.dtype == torch.float32:
        return N.KV_MIXED
    raise TypeError(f"v and x must be float64 (FP64 path) or float32 (mixed path), got {t.dtype}")


def _check_pair(v: torch.Tensor, x: torch.Tensor):
    if not (isinstance(v, torch.Tensor) and isinstance(x, torch.Tensor)):
        raise TypeError("v and x must be torch tensors")
    if not (v.is_cuda and x.is_cuda):
        raise ValueError("v and x must be CUDA tensors (this library has no CPU path)")
    if v.dtype != x.dtype:
        raise TypeError("v and x must have the same dtype")
    if v.shape != x.shape:
        raise ValueError("v and x must have the same shape")
    return v.contiguous(), x.contiguous(), _dtype_code(v)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def kv_log(v, x, bins: int = 0):
    """log K_v(x) elementwise (Algorithm 3 with Eq. int)."""
    v, x, dt = _check_pair(v, x)
    out = torch.empty_like(v)
    b = bins or (128 if dt == N.KV_F64 else 40)
    N.check(N.lib().kv_log(_ptr(v), _ptr(x), _ptr(out), v.numel(), b, dt, _stream_ptr(v.device)), "kv_log")
    return out


def kv_log_dv(v, x, bins: int = 0):
    """d/dv log K_v(x) elementwise (Sec. 4.1)."""
    v, x, dt = _check_pair(v, x)
    out = torch.empty_like(v)
    b = bins or (128 if dt == N.KV_F64 else 40)
    N.check(N.lib().kv_log_dv(_ptr(v), _ptr(x), _ptr(out), v.numel(), b, dt, _stream_ptr(v.device)),
            "kv_log_dv")
    return out


def kv_log_dx(v, x, bins: int = 0):
    """d/dx log K_v(x) elementwise (Sec. 4.1)."""
    v, x, dt = _check_pair(v, x)
    out = torch.empty_like(v)
    b = bins or (128 if dt == N.KV_F64 else 40)
    N.check(N.lib().kv_log_dx(_ptr(v), _ptr(x), _ptr(out), v.numel(), b, dt, _stream_ptr(v.device)),
            "kv_log_dx")
    return out


def kv_fwd_bwd(v, x, bins: int = 0):
    """(log K, d/dv log K, d/dx log K) from one pass over the bins."""
    v, x, dt = _check_pair(v, x)
    lk = torch.empty_like(v)
    dv = torch.empty_like(v)
    dx = torch.empty_like(v)
    b = bins or (128 if dt == N.KV_F64 else 40)
    N.check(N.lib().kv_fwd_bwd(_ptr(v), _ptr(x), _ptr(lk), _ptr(dv), _ptr(dx), v.numel(), b, dt,
                               _stream_ptr(v.device)), "kv_fwd_bwd")
    return lk, dv, dx


def kv_fwd_bwd_ex(v, x, *, bins: int = 0, bracket: str = "plain", log_eps: float = 0.0,
                  max_iter: int = 0, lanes: int = 0, mlp=None, grad_out=None,
                  want=("logk", "dv", "dx"), status: bool = False, fallback_count=None,
                  out=None, second: bool = False, analytic_peak_start: bool = False):
    """The general call (kv_fwd_bwd_ex).  Returns a dict with the requested outputs and, with
    ``status=True``, the per-pair status bytes; ``second=True`` adds the second derivatives
    ``d2v``, ``dvx``, ``d2x`` (Sec. 4.1, n + m = 2).  ``out`` may supply preallocated tensors.
    ``analytic_peak_start=True`` sets KV_FLAG_PEAK_ANALYTIC_START (the FP64 bracket's peak search
    on [0, asinh(v/x)] instead of Algorithm 1's doublings)."""
    v, x, dt = _check_pair(v, x)
    out = dict(out or {})
    want = tuple(want) + (("d2v", "dvx", "d2x") if second else ())
    for k in want:
        if k not in out:
            out[k] = torch.empty_like(v)
    if status and "status" not in out:
        out["status"] = torch.empty(v.shape, dtype=torch.uint8, device=v.device)
    a = N.KvArgs()
    a.v, a.x = v.data_ptr(), x.data_ptr()
    a.logk = out["logk"].data_ptr() if "logk" in want else None
    a.dv = out["dv"].data_ptr() if "dv" in want else None
    a.dx = out["dx"].data_ptr() if "dx" in want else None
    if grad_out is not None:
        grad_out = grad_out.contiguous()
        if grad_out.dtype != v.dtype or grad_out.shape != v.shape or not grad_out.is_cuda:
            raise ValueError("grad_out must match v in dtype, shape and device")
        a.grad_out = grad_out.data_ptr()
    a.n = v.numel()
    a.bins = bins
    a.dtype = dt
    a.bracket = {"plain": N.KV_BRACKET_PLAIN, "mlp": N.KV_BRACKET_MLP, "f32": N.KV_BRACKET_PLAIN_F32}[bracket]
    a.log_eps = log_eps
    a.max_iter = max_iter
    a.lanes = lanes
    a.mlp = mlp.handle if mlp is not None else None
    a.status = out["status"].data_ptr() if status else None
    a.fallback_count = fallback_count.data_ptr() if fallback_count is not None else None
    a.stream = _stream_ptr(v.device)
    if second:
        a.d2v, a.dvx, a.d2x = (out[k].data_ptr() for k in ("d2v", "dvx", "d2x"))
    a.flags = N.KV_FLAG_PEAK_ANALYTIC_START if analytic_peak_start else 0
    N.check(N.lib().kv_fwd_bwd_ex(ctypes.byref(a)), "kv_fwd_bwd_ex")
    return out


HOST_TRANSFER = {"auto": N.KV_HOST_AUTO, "staged": N.KV_HOST_STAGED, "direct": N.KV_HOST_DIRECT}


def kv_fwd_bwd_host(v, x, *, bins: int = 0, bracket: str = "plain", mlp=None, log_eps: float = 0.0,
                    out=None, transfer: str = "auto"):
    """kv_fwd_bwd_ex on host numpy arrays; returns (logk, dv, dx) numpy arrays.  `transfer`:
    "staged" copies through device buffers (any host memory; pinned gives full copy speed),
    "direct" lets the kernels read and write the host buffers in place (all five must be pinned
    and mapped, e.g. numpy views of torch pin_memory() tensors), "auto" takes "direct" for such
    buffers on a coherent CPU-GPU link (see host_direct_supported) and "staged" otherwise."""
    import numpy as np
    v = np.ascontiguousarray(v)
    x = np.ascontiguousarray(x)
    if v.dtype != x.dtype or v.shape != x.shape:
        raise ValueError("v and x must have the same dtype and shape")
    if v.dtype == np.float64:
        dt = N.KV_F64
    elif v.dtype == np.float32:
        dt = N.KV_MIXED
    else:
        raise TypeError("host arrays must be float64 or float32")
    if transfer not in HOST_TRANSFER:
        raise ValueError(f"transfer must be one of {sorted(HOST_TRANSFER)}")
    if out is None:
        out = tuple(np.empty_like(v) for _ in range(3))
    lk, dv, dx = out
    a = N.KvArgs()
    a.v, a.x = v.ctypes.data, x.ctypes.data
    a.logk, a.dv, a.dx = lk.ctypes.data, dv.ctypes.data, dx.ctypes.data
    a.n = v.size
    a.bins = bins
    a.dtype = dt
    a.bracket = {"plain": N.KV_BRACKET_PLAIN, "mlp": N.KV_BRACKET_MLP, "f32": N.KV_BRACKET_PLAIN_F32}[bracket]
    a.log_eps = log_eps
    a.mlp = mlp.handle if mlp is not None else None
    a.stream = _stream_ptr(torch.device("cuda", torch.cuda.current_device()))
    N.check(N.lib().kv_fwd_bwd_host_ex(ctypes.byref(a), HOST_TRANSFER[transfer]), "kv_fwd_bwd_host_ex")
    return lk, dv, dx


def debug_set_wait_limit(iterations: int) -> int:
    """Test hook for the fast path's failure handling: the iteration limit of its bounded wait for
    the tensor-core results (0: give up at once, so every CTA hands its pairs to the fallback
    pass; < 0: the default).  Returns the previous setting (-1 = default)."""
    return int(N.lib().kv_debug_set_wait_limit(int(iterations)))


def debug_set_end_terms(on: bool) -> int:
    """Test hook for the fast path's bins: whether bin n's trapezoid terms come from the range
    check's evaluation of the right end (the default) or are computed as one of the bins.
    Returns the previous setting (1 = on)."""
    return int(N.lib().kv_debug_set_end_terms(1 if on else 0))


def trim_memory() -> None:
    """Release the device memory the library's scratch pool keeps reserved between calls."""
    N.check(N.lib().kv_trim_memory(), "kv_trim_memory")


def host_direct_supported() -> bool:
    """Whether the current GPU reaches host memory over a coherent link (NVLink-C2C class), the
    condition under which transfer="auto" reads and writes pinned host buffers in place."""
    return bool(N.lib().kv_host_direct_supported())


def kv_bracket(v, x, log_eps: float = 0.0, max_iter: int = 0):
    """The plain bracket (Algorithms 1-3): float64 tensors t0, t_p, t1, g(t_p)."""
    v, x, dt = _check_pair(v, x)
    outs = [torch.empty(v.shape, dtype=torch.float64, device=v.device) for _ in range(4)]
    N.check(N.lib().kv_bracket(_ptr(v), _ptr(x), *[_ptr(o) for o in outs], v.numel(), dt, log_eps,
                               max_iter, _stream_ptr(v.device)), "kv_bracket")
    return tuple(outs)


def kv_grad(grad_out, dv, dx):
    """The backward epilogue: (grad_out * dv, grad_out * dx)."""
    dt = _dtype_code(dv)
    gv = torch.empty_like(dv)
    gx = torch.empty_like(dx)
    grad_out = grad_out.contiguous()
    N.check(N.lib().kv_grad(_ptr(grad_out), _ptr(dv.contiguous()), _ptr(dx.contiguous()), _ptr(gv),
                            _ptr(gx), dv.numel(), dt, _stream_ptr(dv.device)), "kv_grad")
    return gv, gx


def kv_sum(a):
    """Deterministic sum of all elements as a float64 CUDA scalar tensor."""
    if not a.is_cuda:
        raise ValueError("kv_sum needs a CUDA tensor")
    a = a.contiguous()
    dt = _dtype_code(a)
    out = torch.empty((), dtype=torch.float64, device=a.device)
    N.check(N.lib().kv_sum(_ptr(a), a.numel(), dt, _ptr(out), _stream_ptr(a.device)), "kv_sum")
    return out


def kv_grad2(go, gg_v, gg_x, dv, dx, d2v, dvx, d2x):
    """The second backward pass's epilogue: (go (gg_v d2v + gg_x dvx), go (gg_v dvx + gg_x d2x),
    gg_v dv + gg_x dx); gg_v or gg_x may be None (zero)."""
    dt = _dtype_code(dv)
    outs = [torch.empty_like(dv) for _ in range(3)]
    c = lambda t: None if t is None else t.contiguous()
    N.check(N.lib().kv_grad2(_ptr(c(go)), _ptr(c(gg_v)), _ptr(c(gg_x)), _ptr(c(dv)), _ptr(c(dx)),
                             _ptr(c(d2v)), _ptr(c(dvx)), _ptr(c(d2x)), *[_ptr(o) for o in outs],
                             dv.numel(), dt, _stream_ptr(dv.device)), "kv_grad2")
    return tuple(outs)


class _LogBesselKGrad(torch.autograd.Function):
    """(go * d/dv log K, go * d/dx log K) as a function of (v, x, go), so that the gradient of
    log_besselk is itself differentiable (Hessian-vector products, double backward).  Its backward
    asks the library for the second derivatives from the same bins and range."""

    @staticmethod
    def forward(ctx, v, x, go, dv, dx, bins, bracket, mlp):
        ctx.save_for_backward(v, x, go, dv, dx)
        ctx.cfg = (bins, bracket, mlp)
        return kv_grad(go.contiguous(), dv, dx)

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gg_v, gg_x):
        v, x, go, dv, dx = ctx.saved_tensors
        bins, bracket, mlp = ctx.cfg
        s = kv_fwd_bwd_ex(v.detach(), x.detach(), bins=bins, bracket=bracket, mlp=mlp, want=(),
                          second=True)
        ov, ox, ogo = kv_grad2(go, gg_v, gg_x, dv, dx, s["d2v"], s["dvx"], s["d2x"])
        return ov, ox, ogo, None, None, None, None, None


class _LogBesselK(torch.autograd.Function):
    """log K_v(x) with the fused backward: the forward keeps d/dv and d/dx from the same bins
    and bracket; the backward multiplies them by the incoming gradient (no re-integration), and
    is itself differentiable once more through _LogBesselKGrad."""

    @staticmethod
    def forward(ctx, v, x, bins, bracket, mlp):
        vc, xc, _ = _check_pair(v.detach(), x.detach())
        want = ("logk", "dv", "dx") if (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]) else ("logk",)
        out = kv_fwd_bwd_ex(vc, xc, bins=bins, bracket=bracket, mlp=mlp, want=want)
        if len(want) == 3:
            # the inputs themselves (not detached copies): a double backward differentiates
            # the gradient with respect to them
            ctx.save_for_backward(v, x, out["dv"], out["dx"])
        ctx.cfg = (bins, bracket, mlp)
        return out["logk"]

    @staticmethod
    def backward(ctx, grad):
        v, x, dv, dx = ctx.saved_tensors
        if torch.is_grad_enabled():  # create_graph: keep the gradient differentiable
            gv, gx = _LogBesselKGrad.apply(v, x, grad, dv, dx, *ctx.cfg)
        else:
            gv, gx = kv_grad(grad.contiguous(), dv, dx)
        return gv, gx, None, None, None


def log_besselk(v, x, bins: int = 0, bracket: str = "plain", mlp=None):
    """Differentiable log K_v(x) (autograd through the library's fused backward)."""
    return _LogBesselK.apply(v, x, bins, bracket, mlp)
