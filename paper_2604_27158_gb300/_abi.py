"""ctypes binding of liblbmfno.so: the C ABI of include/lbmfno.h under the same names.

Argument marshalling only.  Every computation runs in the library's CUDA
kernels; there is no CPU or PyTorch fallback, and loading fails loudly when the
library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

# enum lbm_status
LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, LBM_ERR_UNSUPPORTED = range(6)
# enum lbm_bc
LBM_BC_PERIODIC, LBM_BC_PRESSURE, LBM_BC_VELOCITY = 0, 1, 2
LBM_NSTAT = 8
(LBM_STAT_RESIDUAL, LBM_STAT_UNORM, LBM_STAT_DP, LBM_STAT_MASS, LBM_STAT_MOMX, LBM_STAT_MOMY,
 LBM_STAT_BAD, LBM_STAT_FLUID) = range(8)


class LbmError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed with status {code}: {msg}")
        self.code = code


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("tau", ctypes.c_double),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("bc_west", ctypes.c_int32), ("bc_east", ctypes.c_int32),
                ("west_value", ctypes.c_double), ("east_value", ctypes.c_double)]


class lbm_layout(ctypes.Structure):
    _fields_ = [("f_elems", ctypes.c_size_t), ("mask_words", ctypes.c_size_t),
                ("cells", ctypes.c_size_t), ("ws_bytes", ctypes.c_size_t)]


VP = ctypes.c_void_p
I = ctypes.c_int
_PROTOS = {
    "lbm_last_error": ([], ctypes.c_char_p),
    "lbm_query_layout": ([ctypes.POINTER(lbm_grid), I, ctypes.POINTER(lbm_layout)], I),
    "lbm_init": ([ctypes.POINTER(lbm_grid), I, VP, VP, VP, VP, ctypes.c_double, VP,
                  ctypes.POINTER(VP)], I),
    "lbm_step": ([VP, I, VP], I),
    "lbm_macro": ([VP, VP, VP, VP, VP], I),
    "lbm_residual": ([VP, ctypes.POINTER(ctypes.c_double), I, VP], I),
    "lbm_reinit_from_macro": ([VP, VP, VP, VP, I, VP], I),
    "lbm_export_f": ([VP, VP, VP], I),
    "lbm_set_state": ([VP, VP, VP], I),
    "lbm_get_state": ([VP, VP, VP], I),
    "lbm_steps_done": ([VP, ctypes.POINTER(ctypes.c_longlong)], I),
    "lbm_destroy": ([VP], I),
}


def declared_symbols():
    """Function names the ABI header declares (parsed from include/*.h)."""
    import re
    inc = os.path.join(os.path.dirname(_build.PKG), "include")
    names = []
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            names += re.findall(r"^\s*(?:int|const char\s*\*)\s+(\w+)\s*\(", txt, flags=re.M)
    return names


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            handle = ctypes.CDLL(path)
            for name, (args, res) in _PROTOS.items():
                fn = getattr(handle, name)
                fn.argtypes = args
                fn.restype = res
            _lib = handle
    return _lib


def last_error() -> str:
    return lib().lbm_last_error().decode(errors="replace")


def check(fn: str, code: int) -> None:
    if code != LBM_OK:
        raise LbmError(fn, code, last_error())


def call(name: str, *args) -> None:
    check(name, getattr(lib(), name)(*args))
