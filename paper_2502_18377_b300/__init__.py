"""B300-native (sm_103a) batched NeuRLP-PDE solver of Mechanistic PDE Networks.

The compute path is libmpn.so (CUDA kernels behind the C ABI of
include/mpn.h); this package holds its ctypes binding, a
torch.autograd.Function over it, and the seeded synthetic workloads.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "binding", "autograd"]
