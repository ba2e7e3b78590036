"""GB300-native geodesic ray tracer after MALBEC (arXiv:1803.08320).

The compute path is libmalbec.so (hand-written CUDA for sm_103a, C ABI in
include/malbec.h); `malbec` is its thin Python binding and `workloads` holds
the seeded synthetic inputs.
"""
from . import malbec, workloads  # noqa: F401

__all__ = ["malbec", "workloads"]
