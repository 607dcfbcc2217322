"""CPU oracle for batched log K_v(x), d/dv log K and d/dx log K (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product path (the CUDA library and its binding) never does,
and the two share no code.

* :func:`o1` -- the paper's fixed-bin integration method (Sec. 2, Algorithms 1-3, Eq. (int),
  Sec. 4.1 derivatives) in FP64 (``precision="double"``) or, with the same steps, in
  ``long double`` (``precision="long"``).
* :func:`dense` -- the integral of Eq. (1)-(2) by adaptive Gauss-Legendre quadrature in
  ``long double`` (the truth the method is measured against).
* :mod:`oracle.mlp` -- the learned bracket's MLP forward/backward/Adam in float64 numpy.

The C source is compiled on first use (or by :func:`build`) with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS: dict[str, ctypes.CDLL] = {}
_LOCK = threading.Lock()

#: log of the FP64 machine epsilon 2^-52 (Sec. 2.1: the range keeps f >= eps * f(t_p)).
LOG_EPS_F64 = -52.0 * math.log(2.0)
#: log of the FP32 machine epsilon 2^-23.
LOG_EPS_F32 = -23.0 * math.log(2.0)
#: Algorithm 2's iteration cap (tol = 1, max_iter = 10 in the paper).
MAX_ITER = 10
#: cap on the doublings of Algorithm 1 (t up to 2^12 above the start covers every finite double).
MAX_RANGE = 11

_VARIANTS = {
    "double": ("libkv_oracle_d.so", ["-DKV_REAL=double", "-DKV_SUFFIX=d"]),
    "long": ("libkv_oracle_ld.so", ["-DKV_REAL=long double", "-DKV_SUFFIX=ld", "-DKV_DENSE"]),
}


def _compile(name: str, defines: list[str]) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, name)
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", *defines, _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build() -> None:
    """Compile both variants of the oracle library (idempotent)."""
    for key in _VARIANTS:
        _lib(key)


def compile_variant_source(src_path: str, out_dir: str) -> dict:
    """Compile another copy of the oracle source (both precisions) into out_dir and return the
    loaded libraries, for tests that plant mistakes in a copy and check that the pins catch
    them.  Use with `swap_libraries`."""
    libs = {}
    for key, (name, defines) in _VARIANTS.items():
        out = os.path.join(out_dir, name)
        subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", *defines, src_path,
                        "-o", out, "-lm"], check=True)
        libs[key] = out
    return libs


class swap_libraries:
    """Context manager: the oracle functions use the given compiled copies instead of the
    package's own library (test infrastructure for planted-mistake checks)."""

    def __init__(self, paths: dict):
        self.paths = paths
        self.saved = None

    def __enter__(self):
        with _LOCK:
            self.saved = dict(_LIBS)
        build()
        saved_compile = globals()["_compile"]
        try:
            globals()["_compile"] = lambda name, defines: self.paths["long" if "ld" in name else "double"]
            with _LOCK:
                _LIBS.clear()
            for key in _VARIANTS:
                _lib(key)
        finally:
            globals()["_compile"] = saved_compile
        return self

    def __exit__(self, *exc):
        with _LOCK:
            _LIBS.clear()
            _LIBS.update(self.saved)


def _lib(precision: str) -> ctypes.CDLL:
    with _LOCK:
        if precision not in _LIBS:
            name, defines = _VARIANTS[precision]
            path = _compile(name, defines)
            lib = ctypes.CDLL(path)
            sfx = "d" if precision == "double" else "ld"
            P = ctypes.c_void_p
            f = getattr(lib, f"kv_oracle_o1_{sfx}")
            f.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                          ctypes.c_double, ctypes.c_int, P, P, P, P, P, ctypes.c_int]
            f.restype = None
            f = getattr(lib, f"kv_oracle_g_{sfx}")
            f.argtypes = [ctypes.c_double, ctypes.c_double, P, ctypes.c_int64, P, P, P]
            f.restype = None
            f = getattr(lib, f"kv_oracle_alg12_{sfx}")
            f.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int, ctypes.c_int, P]
            f.restype = None
            if precision == "long":
                lib.kv_oracle_dense.argtypes = [P, P, ctypes.c_int64, P, P, P, P, ctypes.c_int]
                lib.kv_oracle_dense.restype = None
            _LIBS[precision] = lib
        return _LIBS[precision]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())


def o1(v, x, bins: int = 128, log_eps: float = LOG_EPS_F64, max_iter: int = MAX_ITER,
       tol: float = 0.0, max_range: int = MAX_RANGE, precision: str = "double",
       threads: int = 0, bracket: bool = False, second: bool = False) -> dict:
    """The fixed-bin method (Algorithm 3) on arrays of (v, x).

    Returns a dict of float64 arrays ``logk``, ``dv``, ``dx``; with ``bracket=True`` also
    ``t0``, ``tp``, ``t1``, ``G`` (= g(t_p)); with ``second=True`` also the second derivatives
    of log K, ``d2v`` (d2/dv2), ``dvx`` (d2/dv dx) and ``d2x`` (d2/dx2), from the same bins
    (Sec. 4.1).  ``threads=0`` uses every host core.
    """
    v = _as_f64(v)
    x = _as_f64(x)
    if v.shape != x.shape:
        raise ValueError("v and x must have the same number of elements")
    if bins < 1:
        raise ValueError("bins must be >= 1")
    n = v.size
    logk = np.empty(n)
    dv = np.empty(n)
    dx = np.empty(n)
    brk = np.empty(4 * n) if bracket else None
    d2 = np.empty(3 * n) if second else None
    lib = _lib(precision)
    sfx = "d" if precision == "double" else "ld"
    getattr(lib, f"kv_oracle_o1_{sfx}")(
        _ptr(v), _ptr(x), n, bins, log_eps, max_iter, tol, max_range, _ptr(logk), _ptr(dv),
        _ptr(dx), _ptr(brk) if bracket else None, _ptr(d2) if second else None, threads)
    out = {"logk": logk, "dv": dv, "dx": dx}
    if bracket:
        b = brk.reshape(n, 4)
        out.update(t0=b[:, 0].copy(), tp=b[:, 1].copy(), t1=b[:, 2].copy(), G=b[:, 3].copy())
    if second:
        d = d2.reshape(n, 3)
        out.update(d2v=d[:, 0].copy(), dvx=d[:, 1].copy(), d2x=d[:, 2].copy())
    return out


def dense(v, x, threads: int = 0, second: bool = False) -> dict:
    """log K, d/dv log K, d/dx log K (and with ``second=True`` d2v, dvx, d2x) by adaptive
    Gauss-Legendre quadrature in long double."""
    v = _as_f64(v)
    x = _as_f64(x)
    n = v.size
    logk = np.empty(n)
    dv = np.empty(n)
    dx = np.empty(n)
    d2 = np.empty(3 * n) if second else None
    _lib("long").kv_oracle_dense(_ptr(v), _ptr(x), n, _ptr(logk), _ptr(dv), _ptr(dx),
                                 _ptr(d2) if second else None, threads)
    out = {"logk": logk, "dv": dv, "dx": dx}
    if second:
        d = d2.reshape(n, 3)
        out.update(d2v=d[:, 0].copy(), dvx=d[:, 1].copy(), d2x=d[:, 2].copy())
    return out


def g_eval(v: float, x: float, t, precision: str = "double"):
    """g, g', g'' of Sec. 2.1 at the points t."""
    t = _as_f64(t)
    g = np.empty_like(t)
    gp = np.empty_like(t)
    gpp = np.empty_like(t)
    sfx = "d" if precision == "double" else "ld"
    getattr(_lib(precision), f"kv_oracle_g_{sfx}")(v, x, _ptr(t), t.size, _ptr(g), _ptr(gp), _ptr(gpp))
    return g, gp, gpp


def alg12(v: float, x: float, kind: int, t_start: float, t_neg: float, t_pos: float,
          G: float = 0.0, log_eps: float = LOG_EPS_F64, max_iter: int = MAX_ITER,
          max_range: int = MAX_RANGE, precision: str = "double"):
    """Algorithm 1 from ``t_start`` and Algorithm 2 on (t_neg, t_pos) for F = g' (kind 0)
    or F = g - G - log eps (kind 1).  Returns (range_pos_end, range_neg_end, zero)."""
    out = np.empty(3)
    sfx = "d" if precision == "double" else "ld"
    getattr(_lib(precision), f"kv_oracle_alg12_{sfx}")(
        v, x, G, log_eps, kind, t_start, t_neg, t_pos, max_iter, max_range, _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def host_cores() -> int:
    """Threads the oracle's OpenMP loops use by default."""
    return os.cpu_count() or 1
