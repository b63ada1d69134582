"""GB300-native space-time fast-diagonalisation solver for the linear Schroedinger equation.

The compute path is the CUDA library libstfdm.so (C ABI in include/stfdm.h),
built in-tree for sm_103a; `stfdm` is its thin ctypes binding and `autograd`
wraps the solve and its adjoint in a torch.autograd.Function.
"""
from . import stfdm  # noqa: F401

__all__ = ["stfdm"]
