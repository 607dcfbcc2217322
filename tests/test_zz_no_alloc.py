"""kv_sum_noalloc: the sum for callers that cannot allocate device memory.

Some callers have all of their device memory reserved up front (a framework's caching
allocator, or a fixed budget), so a library call must not allocate any.  kv_sum_noalloc keeps
its partial sums in a fixed device array inside the library instead of allocating them.  This
file checks it, through the C ABI, against kv_sum on the same inputs, twice in a row (the second
call reuses the array the first one left behind).  It is collected last so that a stop at the
first failure has run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2108_11560_gb300 import _native as N

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _sum(fn, t, dtype_code):
    out = torch.full((), float("nan"), dtype=torch.float64, device=DEV)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    rc = fn(ctypes.c_void_p(t.data_ptr()), t.numel(), dtype_code, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(stream))
    assert rc == 0, N.lib().kv_strerror(rc)
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("n, dtype", [(3_000_001, torch.float64), (1_234_567, torch.float32),
                                      (10_000_019, torch.float64), (1, torch.float64)])
def test_no_alloc_sum_matches_kv_sum_twice(n, dtype):
    lib = N.lib()
    code = N.KV_F64 if dtype == torch.float64 else N.KV_MIXED
    a = torch.from_numpy(np.random.default_rng(n).standard_normal(n)).to(DEV, dtype)
    b = torch.from_numpy(np.random.default_rng(n + 1).standard_normal(n)).to(DEV, dtype)
    scale = float(a.double().abs().sum().item()) + 1.0
    ref_a = _sum(lib.kv_sum, a, code)
    ref_b = _sum(lib.kv_sum, b, code)
    # two calls in a row on different data: the second must not see the first one's partials
    got_a = _sum(lib.kv_sum_noalloc, a, code)
    got_b = _sum(lib.kv_sum_noalloc, b, code)
    assert abs(got_a - ref_a) <= 1e-12 * scale
    assert abs(got_b - ref_b) <= 1e-12 * scale
    if n <= 4_194_304:
        assert got_a == ref_a and got_b == ref_b  # same blocking, same order


def test_no_alloc_sum_empty_and_limits():
    lib = N.lib()
    empty = torch.zeros(0, dtype=torch.float64, device=DEV)
    out = torch.full((), 5.0, dtype=torch.float64, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    assert lib.kv_sum_noalloc(ctypes.c_void_p(empty.data_ptr() or 256), 0, N.KV_F64,
                              ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    assert out.item() == 0.0
    fake = ctypes.c_void_p(256)
    # beyond the array's capacity: rejected on the host, before any GPU work
    assert lib.kv_sum_noalloc(fake, N.KV_SUM_NOALLOC_MAX_N + 1, N.KV_F64, fake, stream) == -2
    assert lib.kv_sum_noalloc(fake, -1, N.KV_F64, fake, stream) == -2
    assert lib.kv_sum_noalloc(fake, 10, 9, fake, stream) == -4
