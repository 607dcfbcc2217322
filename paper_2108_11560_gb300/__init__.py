"""Batched log K_v(x) and its derivatives in v and x on GB300 (sm_103a).

The fixed-bin integration method of arXiv 2108.11560 behind a C ABI (include/kv.h) with a thin
PyTorch binding.  ``paper_2108_11560_gb300.kv`` holds the binding; importing this package does
not load the CUDA library (``workloads`` stays usable without a GPU).
"""

__all__ = ["kv", "workloads", "build"]
