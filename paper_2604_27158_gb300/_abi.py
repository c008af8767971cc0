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
LBM_STEP_VARIANTS = 6
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


class fno_config(ctypes.Structure):
    _fields_ = [("c_in", ctypes.c_int32), ("c_out", ctypes.c_int32), ("width", ctypes.c_int32),
                ("layers", ctypes.c_int32), ("modes", ctypes.c_int32),
                ("dec_layers", ctypes.c_int32), ("dec_size", ctypes.c_int32),
                ("activation", ctypes.c_int32), ("padding", ctypes.c_int32)]


class fno_sizes(ctypes.Structure):
    _fields_ = [("n_params", ctypes.c_size_t), ("packed_bytes", ctypes.c_size_t),
                ("ws_bytes", ctypes.c_size_t)]


class fno_train_sizes(ctypes.Structure):
    _fields_ = [("n_params", ctypes.c_size_t), ("saved_bytes", ctypes.c_size_t),
                ("ws_bytes", ctypes.c_size_t)]


class hybrid_config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("use_fno", ctypes.c_int32), ("neq_mode", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("k_lbm", ctypes.c_int32), ("m_fno", ctypes.c_int32),
                ("rho_lo", ctypes.c_double), ("rho_hi", ctypes.c_double),
                ("u_clamp", ctypes.c_double),
                ("in_channels", ctypes.c_int32), ("in_channels_u", ctypes.c_int32)]


class hybrid_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("converged", ctypes.c_int32),
                ("fno_calls", ctypes.c_int32), ("max_residual", ctypes.c_double)]


FNO_ACT_GELU, FNO_ACT_RELU = 0, 1
FNO_PATH_AUTO, FNO_PATH_CUDA_CORES = 0, 1
HYBRID_STEADY, HYBRID_UNSTEADY = 0, 1

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
    "lbm_step_residual": ([VP, ctypes.POINTER(ctypes.c_double), I, VP], I),
    "lbm_stream_probe": ([VP, I, VP], I),
    "lbm_set_persistent": ([VP, I], I),
    "lbm_barrier_selftest": ([VP, VP, I, ctypes.c_double, VP], I),
    "lbm_reinit_from_macro": ([VP, VP, VP, VP, I, VP], I),
    "lbm_export_f": ([VP, VP, VP], I),
    "lbm_vorticity": ([VP, VP, VP, VP, VP], I),
    "lbm_set_state": ([VP, VP, VP], I),
    "lbm_get_state": ([VP, VP, VP], I),
    "lbm_steps_done": ([VP, ctypes.POINTER(ctypes.c_longlong)], I),
    "lbm_autotune": ([VP, I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(I), VP], I),
    "lbm_set_step_variant": ([VP, I], I),
    "lbm_get_step_variant": ([VP, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                              ctypes.POINTER(I)], I),
    "lbm_destroy": ([VP], I),
    "lbm_wait_selftest": ([VP, I, ctypes.c_double, VP], I),
    "lbm_adjoint_macro": ([VP, VP, VP, VP, VP, VP, VP], I),
    "lbm_adjoint_step": ([VP, VP, VP, VP, VP], I),
    "lbm_adjoint_reinit": ([VP, VP, VP, VP, VP, I, VP, VP, VP, VP, VP], I),
    "fno_query": ([ctypes.POINTER(fno_config), I, I, I, ctypes.POINTER(fno_sizes)], I),
    "fno_create": ([ctypes.POINTER(fno_config), VP, VP, VP, ctypes.POINTER(VP)], I),
    "fno_forward": ([VP, VP, VP, I, I, I, VP, ctypes.c_size_t, VP], I),
    "fno_get_config": ([VP, ctypes.POINTER(fno_config)], I),
    "fno_set_path": ([VP, I], I),
    "fno_uses_tensor_cores": ([VP, I, I, ctypes.POINTER(I)], I),
    "fno_check": ([VP, VP, I, I, I, VP], I),
    "fno_activation_eval": ([I, VP, VP, ctypes.c_size_t, VP], I),
    "fno_destroy": ([VP], I),
    "fno_train_query": ([ctypes.POINTER(fno_config), I, I, I, ctypes.POINTER(fno_train_sizes)], I),
    "fno_train_forward": ([ctypes.POINTER(fno_config), VP, VP, VP, I, I, I, VP, VP, VP], I),
    "fno_train_backward": ([ctypes.POINTER(fno_config), VP, VP, VP, VP, VP, I, I, I, VP, VP], I),
    "hybrid_query_ws": ([ctypes.POINTER(lbm_grid), I, ctypes.POINTER(fno_config),
                         ctypes.POINTER(fno_config), ctypes.POINTER(ctypes.c_size_t)], I),
    "hybrid_create": ([VP, VP, VP, ctypes.POINTER(hybrid_config), VP, ctypes.c_size_t,
                       ctypes.POINTER(VP)], I),
    "hybrid_advance": ([VP, I, ctypes.POINTER(hybrid_stats), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_double), VP], I),
    "hybrid_destroy": ([VP], I),
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
