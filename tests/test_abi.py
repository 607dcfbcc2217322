"""The C-ABI library: it loads, exports every function include/kv.h declares, and rejects bad
arguments on the host before touching the GPU (no compute calls; runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2108_11560_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "kv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(kv_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    return N.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 18
    assert set(names) == set(N.EXPORTED)
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_covers_every_status(lib):
    for code in range(0, -12, -1):
        msg = lib.kv_strerror(code).decode()
        assert msg and msg != "unknown status", code
    assert lib.kv_strerror(-99).decode() == "unknown status"


def test_host_side_argument_errors(lib):
    P = ctypes.c_void_p
    fake = P(256)  # never dereferenced: every call below fails validation first
    # n < 0
    assert lib.kv_log(fake, fake, fake, -1, 32, 0, None) == -2
    # bins out of range
    assert lib.kv_log(fake, fake, fake, 10, 0, 0, None) == -3
    assert lib.kv_fwd_bwd(fake, fake, fake, fake, fake, 10, 4097, 1, None) == -3
    # unknown dtype
    assert lib.kv_log(fake, fake, fake, 10, 32, 7, None) == -4
    # NULL pointers
    assert lib.kv_log(None, fake, fake, 10, 32, 0, None) == -1
    assert lib.kv_fwd_bwd(fake, fake, fake, None, fake, 10, 32, 0, None) == -1
    # misaligned pointer for double
    assert lib.kv_log(P(256 + 4), fake, fake, 10, 32, 0, None) == -5
    # n == 0 is a no-op even with NULL pointers
    assert lib.kv_log(None, None, None, 0, 32, 0, None) == 0
    # extended call: bad log_eps, lanes, MLP bracket without a network or on FP64
    a = N.KvArgs()
    a.v = a.x = a.logk = 256
    a.n, a.bins, a.dtype = 10, 32, 1
    a.log_eps = 1.0
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -7
    a.log_eps = 0.0
    a.lanes = 3
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -7
    a.lanes = 0
    a.bracket = 1
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -8
    a.dtype = 0
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -4
    # bracket / grad / sum validation
    assert lib.kv_bracket(fake, fake, None, None, None, None, 5, 0, 0.0, 0, None) == -1
    assert lib.kv_bracket(fake, fake, fake, None, None, None, 5, 0, 2.0, 0, None) == -7
    assert lib.kv_grad(None, fake, fake, fake, fake, 5, 0, None) == -1
    assert lib.kv_sum(fake, 5, 3, fake, None) == -4
    assert lib.kv_sum(fake, -5, 0, fake, None) == -2
    a = N.KvArgs()
    a.v = a.x = a.logk = a.dv = a.dx = 256
    a.n, a.bins, a.dtype = 5, -1, 0
    assert lib.kv_fwd_bwd_host(ctypes.byref(a)) == -3
    a.bins = 0
    a.status = 256
    assert lib.kv_fwd_bwd_host(ctypes.byref(a)) == -7
    a.status = None
    assert lib.kv_fwd_bwd_host_ex(ctypes.byref(a), 3) == -7  # no such transfer mode
    assert lib.kv_fwd_bwd_host_ex(ctypes.byref(a), -1) == -7
    assert lib.kv_fwd_bwd_host_ex(None, 0) == -1


def test_second_derivative_argument_errors(lib):
    P = ctypes.c_void_p
    fake = P(256)
    a = N.KvArgs()
    a.v = a.x = 256
    a.n, a.bins, a.dtype = 10, 32, 0
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -1  # no output at all
    a.d2x = 256 + 4  # misaligned for double
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -5
    # the host-buffer call takes no second-derivative outputs
    h = N.KvArgs()
    h.v = h.x = h.logk = 256
    h.n, h.bins, h.dtype = 5, 32, 0
    h.dvx = 256
    assert lib.kv_fwd_bwd_host(ctypes.byref(h)) == -7
    # second backward epilogue
    assert lib.kv_grad2(fake, fake, fake, fake, fake, fake, fake, fake, None, None, None, 5, 0, None) == -1
    assert lib.kv_grad2(None, fake, fake, fake, fake, fake, fake, fake, fake, None, None, 5, 0, None) == -1
    assert lib.kv_grad2(fake, fake, fake, fake, fake, fake, fake, fake, fake, None, None, 5, 9, None) == -4
    assert lib.kv_grad2(fake, fake, fake, fake, fake, fake, fake, fake, fake, None, None, -1, 0, None) == -2


def test_f32_bracket_argument_errors(lib):
    a = N.KvArgs()
    a.v = a.x = a.logk = 256
    a.n, a.bins, a.dtype = 10, 32, 0
    a.bracket = N.KV_BRACKET_PLAIN_F32
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -4  # FP64 I/O has no FP32 bracket
    a.bracket = 3
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -7


def test_flags_argument_errors(lib):
    """kv_args.flags: unknown bits are rejected on the host, before any launch."""
    a = N.KvArgs()
    a.v = a.x = a.logk = 256
    a.n, a.bins, a.dtype = 10, 32, 0
    a.flags = 2
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -7
    a.flags = -1
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -7
    a.flags = N.KV_FLAG_PEAK_ANALYTIC_START
    a.log_eps = 1.0  # the flag itself is valid: the next check (log_eps) reports
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -7
    a.log_eps = 0.0
    a.bins = -1
    assert lib.kv_fwd_bwd_ex(ctypes.byref(a)) == -3
