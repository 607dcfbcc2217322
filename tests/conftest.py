import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs through the C-ABI library)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def rel_logk(a, ref):
    """|a - ref| / max(1, |ref|): the log K error measure (log K crosses 0 where K = 1)."""
    import numpy as np
    return np.abs(np.asarray(a, dtype=np.float64) - ref) / np.maximum(1.0, np.abs(ref))


def rel(a, ref, floor=1e-300):
    """Plain relative error |a - ref| / |ref| (used for d/dv and d/dx)."""
    import numpy as np
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(np.asarray(a, dtype=np.float64) - ref) / np.maximum(np.abs(ref), floor)
