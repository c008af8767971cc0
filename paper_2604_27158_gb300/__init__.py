"""GB300-native (sm_103a) hot path of the hybrid FNO-LBM method (arXiv 2604.27158).

The compute lives in liblbmfno.so (CUDA kernels behind the C ABI declared in
include/lbmfno.h); this package is a thin ctypes front end over it, with
PyTorch used only for device memory and streams.
"""
from . import _abi  # noqa: F401
from ._abi import LbmError, lib  # noqa: F401
from .lbm import BC_PERIODIC, BC_PRESSURE, BC_VELOCITY, GridSpec, Lattice, pack_mask  # noqa: F401
from .fno import Fno, FnoShape, Hybrid, HybridConfig  # noqa: F401

__all__ = ["lib", "LbmError", "GridSpec", "Lattice", "pack_mask", "BC_PERIODIC", "BC_PRESSURE",
           "BC_VELOCITY", "Fno", "FnoShape", "Hybrid", "HybridConfig"]
