"""GB300-native solver for the steady nongray phonon BTE (relaxation-time
approximation, masked Cartesian grid, discrete ordinates).

The compute path is libbte.so (CUDA kernels for sm_103a behind the C ABI of
include/bte.h); ``binding`` marshals arguments to it and ``autograd`` wraps
solve + adjoint in a ``torch.autograd.Function``.  Nothing here computes on
the CPU.
"""
from .binding import (Batch, Plan, BTEError, load, BTE_FP32, BTE_FP64, BTE_OK, BTE_EINVAL,  # noqa: F401
                      BTE_ENOMEM, BTE_ECUDA, BTE_ENOTCONVERGED, BTE_ETIMEOUT, BTE_ENUMERIC, BTE_ESTATE)

__all__ = ["Batch", "Plan", "BTEError", "load", "BTE_FP32", "BTE_FP64", "BTE_OK", "BTE_EINVAL", "BTE_ENOMEM",
           "BTE_ECUDA", "BTE_ENOTCONVERGED", "BTE_ETIMEOUT", "BTE_ENUMERIC", "BTE_ESTATE"]
