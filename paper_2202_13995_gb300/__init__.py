"""GB300-native dense LU solver (the LINPACK hot path of arxiv 2202.13995).

The compute path is the CUDA library `libgb300lu.so` (built from `csrc/` for
sm_103a) behind the C ABI declared in `include/lu.h`; `lu` is its thin ctypes
binding.  `inputs` draws the seeded synthetic workloads.
"""
__all__ = ["inputs", "lu"]
