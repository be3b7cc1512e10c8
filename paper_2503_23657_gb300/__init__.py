"""GB300-native solver for the steady nongray phonon BTE (relaxation-time
approximation, masked Cartesian grid, discrete ordinates).

The compute path is libbte.so (CUDA kernels for sm_103a behind the C ABI of
include/bte.h); ``binding`` marshals arguments to it and ``autograd`` wraps
solve + adjoint in a ``torch.autograd.Function``.  Nothing here computes on
the CPU.
"""
from .binding import Batch, Plan, BTEError, load, BTE_FP32, BTE_FP64  # noqa: F401

__all__ = ["Batch", "Plan", "BTEError", "load", "BTE_FP32", "BTE_FP64"]
