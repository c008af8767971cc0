"""Python front end of the FNO and hybrid calls of the C ABI (fno_*, hybrid_*).

PyTorch supplies device memory and streams; all arithmetic runs in liblbmfno.so.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import call, fno_config, fno_sizes, hybrid_config, hybrid_stats, lbm_grid
from .lbm import Lattice, _stream_ptr


@dataclasses.dataclass(frozen=True)
class FnoShape:
    """Architecture of an FNO (fields of struct fno_config)."""
    c_in: int = 4
    c_out: int = 3
    width: int = 32
    layers: int = 4
    modes: int = 12
    dec_layers: int = 1
    dec_size: int = 32
    activation: int = _abi.FNO_ACT_GELU
    padding: int = 0

    def c(self) -> fno_config:
        return fno_config(self.c_in, self.c_out, self.width, self.layers, self.modes,
                          self.dec_layers, self.dec_size, self.activation, self.padding)


def fno_query(shape: FnoShape, B: int, H: int, W: int) -> fno_sizes:
    out = fno_sizes()
    cfg = shape.c()
    call("fno_query", ctypes.byref(cfg), int(B), int(H), int(W), ctypes.byref(out))
    return out


class Fno:
    """An FNO whose parameters live on one GPU (a thin owner of fno_handle)."""

    def __init__(self, shape: FnoShape, params_flat: np.ndarray, device: str = "cuda",
                 stream=None):
        self.shape = shape
        self.device = torch.device(device)
        sz = fno_query(shape, 1, 2 * shape.modes, 2 * shape.modes + 1)
        flat = np.asarray(params_flat, dtype=np.float32).reshape(-1)
        if flat.size != sz.n_params:
            raise ValueError(f"expected {sz.n_params} parameters, got {flat.size}")
        self.params = torch.from_numpy(flat).to(torch.bfloat16).to(self.device)
        self.packed = torch.empty(sz.packed_bytes, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        cfg = shape.c()
        call("fno_create", ctypes.byref(cfg), self.params.data_ptr(), self.packed.data_ptr(),
             _stream_ptr(stream), ctypes.byref(self._h))
        self._ws: Dict[tuple, torch.Tensor] = {}

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def workspace(self, B: int, H: int, W: int) -> torch.Tensor:
        key = (B, H, W)
        if key not in self._ws:
            n = fno_query(self.shape, B, H, W).ws_bytes
            self._ws[key] = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self._ws[key]

    def forward(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        assert x.dtype == torch.float32 and x.is_contiguous() and x.dim() == 4
        B, cin, H, W = x.shape
        assert cin == self.shape.c_in
        if out is None:
            out = torch.empty((B, self.shape.c_out, H, W), dtype=torch.float32, device=self.device)
        ws = self.workspace(B, H, W)
        call("fno_forward", self._h, x.data_ptr(), out.data_ptr(), B, H, W, ws.data_ptr(),
             ws.numel(), _stream_ptr(stream))
        return out

    __call__ = forward

    def set_path(self, path: int) -> None:
        """FNO_PATH_AUTO (tensor cores where the shape allows) or FNO_PATH_CUDA_CORES."""
        call("fno_set_path", self._h, int(path))

    def uses_tensor_cores(self, H: int, W: int) -> bool:
        v = ctypes.c_int()
        call("fno_uses_tensor_cores", self._h, int(H), int(W), ctypes.byref(v))
        return bool(v.value)

    def check(self, B: int, H: int, W: int, stream=None) -> None:
        """Synchronise and raise if a device-side wait expired in the last forward."""
        ws = self.workspace(B, H, W)
        call("fno_check", self._h, ws.data_ptr(), int(B), int(H), int(W), _stream_ptr(stream))

    def close(self) -> None:
        if self._h:
            _abi.lib().fno_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def activation(x: torch.Tensor, act: int = _abi.FNO_ACT_GELU) -> torch.Tensor:
    """The activation exactly as the tensor-core FNO kernels evaluate it (element-wise,
    FP32, on the device)."""
    assert x.dtype == torch.float32 and x.is_cuda
    x = x.contiguous()
    y = torch.empty_like(x)
    call("fno_activation_eval", int(act), x.data_ptr(), y.data_ptr(), x.numel(), _stream_ptr(None))
    return y


@dataclasses.dataclass
class HybridConfig:
    """Fields of struct hybrid_config."""
    mode: int = _abi.HYBRID_STEADY
    use_fno: int = 1
    neq_mode: int = 1
    check_every: int = 100
    tol: float = 1e-7
    max_steps: int = 200000
    k_lbm: int = 50
    m_fno: int = 5
    rho_lo: float = 0.9
    rho_hi: float = 1.1
    u_clamp: float = 0.2
    in_channels: int = 0    # planes of (rho-1, ux, uy, mask) read by the (density) net, 0 = all
    in_channels_u: int = 0  # planes read by the velocity net, 0 = all

    def c(self) -> hybrid_config:
        return hybrid_config(self.mode, self.use_fno, self.neq_mode, self.check_every, self.tol,
                             self.max_steps, self.k_lbm, self.m_fno, self.rho_lo, self.rho_hi,
                             self.u_clamp, self.in_channels, self.in_channels_u)


class Hybrid:
    """Hybrid FNO-LBM driver over a Lattice and an Fno (a thin owner of hybrid_handle)."""

    def __init__(self, lattice: Lattice, fno: Optional[Fno], cfg: HybridConfig,
                 shape: Optional[FnoShape] = None, fno_u: Optional[Fno] = None):
        """fno: the single network (3 outputs) or, with fno_u, the density network
        (1 output); fno_u: the velocity network (2 outputs)."""
        self.lattice = lattice
        self.fno = fno
        self.fno_u = fno_u
        self.cfg = cfg
        shape = fno.shape if fno is not None else (shape or FnoShape(width=2, layers=1, modes=1,
                                                                      dec_size=1))
        arr = (lbm_grid * len(lattice.grids))(*[g.c() for g in lattice.grids])
        n = ctypes.c_size_t()
        fc = shape.c()
        fcu = fno_u.shape.c() if fno_u is not None else None
        call("hybrid_query_ws", arr, len(lattice.grids), ctypes.byref(fc),
             ctypes.byref(fcu) if fcu is not None else None, ctypes.byref(n))
        self.ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=lattice.device)
        self._h = ctypes.c_void_p()
        hc = cfg.c()
        call("hybrid_create", lattice.handle, fno.handle if fno is not None else None,
             fno_u.handle if fno_u is not None else None, ctypes.byref(hc), self.ws.data_ptr(),
             self.ws.numel(), ctypes.byref(self._h))

    def advance(self, cycles: int = 0, stream=None):
        """Run the steady solve (cycles ignored) or `cycles` unsteady cycles.

        Returns (hybrid_stats, per-grid first-converged step, per-grid residual)."""
        ng = len(self.lattice.grids)
        st = hybrid_stats()
        steps = (ctypes.c_int64 * ng)()
        res = (ctypes.c_double * ng)()
        call("hybrid_advance", self._h, int(cycles), ctypes.byref(st), steps, res,
             _stream_ptr(stream))
        return st, np.array(steps[:], dtype=np.int64), np.array(res[:], dtype=np.float64)

    def close(self) -> None:
        if self._h:
            _abi.lib().hybrid_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
