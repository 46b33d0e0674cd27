"""GB300-native (sm_103a) checkerboard Metropolis for the 2D Ising and
Blume-Capel models (Bisson et al., arXiv 2502.18624).

The compute path is the CUDA library built from csrc/ (C ABI in
include/lat.h); `binding` is its ctypes binding.  Importing this package
loads nothing: the library is loaded on first use of the binding.
"""
from . import _build  # noqa: F401

__all__ = ["binding", "workloads"]
