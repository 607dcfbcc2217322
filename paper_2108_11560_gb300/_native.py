"""ctypes declarations of the C ABI in include/kv.h (libkv.so, built in-tree by build.py).

Loading fails loudly if the library is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_LOCK = threading.Lock()
_LIB = None

# enum values of include/kv.h
KV_F64 = 0
KV_MIXED = 1
KV_BRACKET_PLAIN = 0
KV_BRACKET_MLP = 1
KV_BRACKET_PLAIN_F32 = 2
KV_OK = 0
KV_MAX_BINS = 4096
KV_MLP_NPARAMS = 4482
KV_SUM_NOALLOC_MAX_N = 67108864
KV_PAIR_OK, KV_PAIR_EDGE, KV_PAIR_FALLBACK, KV_PAIR_RANGE_CAP = 0, 1, 2, 4
KV_HOST_AUTO, KV_HOST_STAGED, KV_HOST_DIRECT = 0, 1, 2
KV_FLAG_PEAK_ANALYTIC_START = 1

#: every function include/kv.h declares
EXPORTED = [
    "kv_log", "kv_log_dv", "kv_log_dx", "kv_fwd_bwd", "kv_fwd_bwd_ex", "kv_fwd_bwd_host",
    "kv_fwd_bwd_host_ex", "kv_host_direct_supported", "kv_trim_memory", "kv_debug_set_wait_limit",
    "kv_debug_set_end_terms",
    "kv_bracket", "kv_grad", "kv_grad2", "kv_sum", "kv_sum_noalloc", "kv_mlp_create", "kv_mlp_free", "kv_mlp_save",
    "kv_mlp_load", "kv_mlp_get_params", "kv_mlp_set_params", "kv_mlp_train",
    "kv_mlp_loss_grad", "kv_mlp_predict", "kv_launch_count", "kv_strerror",
    "kv_last_cuda_error",
]


class KvArgs(ctypes.Structure):
    _fields_ = [
        ("v", ctypes.c_void_p), ("x", ctypes.c_void_p), ("logk", ctypes.c_void_p),
        ("dv", ctypes.c_void_p), ("dx", ctypes.c_void_p), ("grad_out", ctypes.c_void_p),
        ("n", ctypes.c_int64), ("bins", ctypes.c_int), ("dtype", ctypes.c_int),
        ("bracket", ctypes.c_int), ("log_eps", ctypes.c_double), ("max_iter", ctypes.c_int),
        ("lanes", ctypes.c_int), ("mlp", ctypes.c_void_p), ("status", ctypes.c_void_p),
        ("fallback_count", ctypes.c_void_p), ("stream", ctypes.c_void_p),
        ("d2v", ctypes.c_void_p), ("dvx", ctypes.c_void_p), ("d2x", ctypes.c_void_p),
        ("flags", ctypes.c_int),
    ]


class KvTrainArgs(ctypes.Structure):
    _fields_ = [
        ("v", ctypes.c_void_p), ("x", ctypes.c_void_p), ("t0", ctypes.c_void_p),
        ("t1", ctypes.c_void_p), ("n", ctypes.c_int64), ("batch", ctypes.c_int),
        ("steps", ctypes.c_int), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float), ("seed", ctypes.c_uint64),
        ("loss_out", ctypes.c_void_p), ("stream", ctypes.c_void_p),
    ]


def _declare(lib):
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "kv_log": [P, P, P, I64, I, I, P],
        "kv_log_dv": [P, P, P, I64, I, I, P],
        "kv_log_dx": [P, P, P, I64, I, I, P],
        "kv_fwd_bwd": [P, P, P, P, P, I64, I, I, P],
        "kv_fwd_bwd_ex": [ctypes.POINTER(KvArgs)],
        "kv_fwd_bwd_host": [ctypes.POINTER(KvArgs)],
        "kv_fwd_bwd_host_ex": [ctypes.POINTER(KvArgs), I],
        "kv_host_direct_supported": [],
        "kv_trim_memory": [],
        "kv_debug_set_wait_limit": [I],
        "kv_debug_set_end_terms": [I],
        "kv_bracket": [P, P, P, P, P, P, I64, I, D, I, P],
        "kv_grad": [P, P, P, P, P, I64, I, P],
        "kv_grad2": [P, P, P, P, P, P, P, P, P, P, P, I64, I, P],
        "kv_sum": [P, I64, I, P, P],
        "kv_sum_noalloc": [P, I64, I, P, P],
        "kv_mlp_create": [ctypes.c_uint64, ctypes.POINTER(P)],
        "kv_mlp_free": [P],
        "kv_mlp_save": [P, ctypes.c_char_p],
        "kv_mlp_load": [ctypes.c_char_p, ctypes.POINTER(P)],
        "kv_mlp_get_params": [P, P, I64],
        "kv_mlp_set_params": [P, P, I64],
        "kv_mlp_train": [P, ctypes.POINTER(KvTrainArgs)],
        "kv_mlp_loss_grad": [P, P, P, P, P, I64, P, P, P],
        "kv_mlp_predict": [P, P, P, P, P, I64, I, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.kv_strerror.argtypes = [ctypes.c_int]
    lib.kv_strerror.restype = ctypes.c_char_p
    lib.kv_launch_count.argtypes = []
    lib.kv_launch_count.restype = ctypes.c_uint64
    lib.kv_last_cuda_error.argtypes = []
    lib.kv_last_cuda_error.restype = ctypes.c_char_p


def lib(build_if_missing: bool = True):
    """The loaded libkv.so (built on first use when nvcc is available)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.LIB
            if build_if_missing and not _build._up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise ImportError(f"libkv.so not found at {path}; run paper_2108_11560_gb300.build")
            # the CUDA runtime PyTorch loaded is the one libkv.so links against
            import torch  # noqa: F401
            handle = ctypes.CDLL(path)
            _declare(handle)
            _LIB = handle
        return _LIB


class KvError(RuntimeError):
    """A non-zero status from the C ABI."""

    def __init__(self, code: int, where: str):
        l = lib(build_if_missing=False)
        msg = l.kv_strerror(code).decode()
        if code == -6:
            msg += ": " + l.kv_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != KV_OK:
        raise KvError(code, where)
