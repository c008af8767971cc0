"""Python front end of the LBM part of the C ABI (lbm_* calls of include/lbmfno.h).

PyTorch supplies device memory and streams; all arithmetic runs in liblbmfno.so.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import call, lbm_grid, lbm_layout

BC_PERIODIC, BC_PRESSURE, BC_VELOCITY = _abi.LBM_BC_PERIODIC, _abi.LBM_BC_PRESSURE, _abi.LBM_BC_VELOCITY


@dataclasses.dataclass
class GridSpec:
    """One lattice of a batch (fields of struct lbm_grid)."""
    nx: int
    ny: int
    tau: float
    fx: float = 0.0
    fy: float = 0.0
    bc_west: int = BC_PERIODIC
    bc_east: int = BC_PERIODIC
    west_value: float = 1.0
    east_value: float = 1.0

    def c(self) -> lbm_grid:
        return lbm_grid(self.nx, self.ny, self.tau, self.fx, self.fy, self.bc_west, self.bc_east,
                        self.west_value, self.east_value)


def pack_mask(solid: np.ndarray) -> np.ndarray:
    """[ny, nx] bool -> uint32 words, ceil(nx/32) per row, bit x%32 = solid(x, y)."""
    solid = np.asarray(solid, dtype=bool)
    ny, nx = solid.shape
    wpr = (nx + 31) // 32
    bits = np.zeros((ny, wpr * 32), dtype=np.uint8)
    bits[:, :nx] = solid
    packed = np.packbits(bits.reshape(ny, wpr, 4, 8), axis=-1, bitorder="little")
    return packed.reshape(ny, wpr, 4).view("<u4").reshape(-1).astype(np.uint32)


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def wait_selftest(arrive: bool, limit_ms: float, device: str = "cuda", stream=None) -> int:
    """Run the library's bounded device-side wait on a barrier that completes (arrive) or
    never does; returns the status code (LBM_OK or LBM_ERR_TIMEOUT) without raising."""
    status = torch.zeros(1, dtype=torch.int32, device=device)
    return int(_abi.lib().lbm_wait_selftest(ctypes.c_void_p(status.data_ptr()), int(arrive),
                                            float(limit_ms), _stream_ptr(stream)))


def query_layout(grids: Sequence[GridSpec]) -> lbm_layout:
    arr = (lbm_grid * len(grids))(*[g.c() for g in grids])
    lay = lbm_layout()
    call("lbm_query_layout", arr, len(grids), ctypes.byref(lay))
    return lay


class Lattice:
    """A batch of D2Q9 lattices resident on one GPU (a thin owner of lbm_handle)."""

    def __init__(self, grids: Sequence[GridSpec], masks: Sequence[np.ndarray], u_max: float = 0.2,
                 device: str = "cuda", stream: Optional[torch.cuda.Stream] = None):
        assert len(grids) == len(masks) and len(grids) > 0
        self.grids: List[GridSpec] = list(grids)
        self.device = torch.device(device)
        self.layout = query_layout(self.grids)
        words = np.concatenate([pack_mask(m) for m in masks])
        assert words.size == self.layout.mask_words
        self.solid = [np.asarray(m, dtype=bool) for m in masks]
        self.mask = torch.from_numpy(words.view(np.int32)).to(self.device)
        self.f_a = torch.empty(self.layout.f_elems, dtype=torch.float32, device=self.device)
        self.f_b = torch.empty(self.layout.f_elems, dtype=torch.float32, device=self.device)
        self.ws = torch.empty(max(self.layout.ws_bytes, 256), dtype=torch.uint8, device=self.device)
        self.cells = int(self.layout.cells)
        offs = [0]
        for g in self.grids:
            offs.append(offs[-1] + g.nx * g.ny)
        self.cell_offsets = offs
        self._h = ctypes.c_void_p()
        arr = (lbm_grid * len(self.grids))(*[g.c() for g in self.grids])
        call("lbm_init", arr, len(self.grids), self.mask.data_ptr(), self.f_a.data_ptr(),
             self.f_b.data_ptr(), self.ws.data_ptr(), float(u_max), _stream_ptr(stream),
             ctypes.byref(self._h))

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def step(self, nsteps: int, stream=None) -> None:
        call("lbm_step", self._h, int(nsteps), _stream_ptr(stream))

    def macro(self, stream=None):
        rho = torch.empty(self.cells, dtype=torch.float32, device=self.device)
        ux = torch.empty_like(rho)
        uy = torch.empty_like(rho)
        call("lbm_macro", self._h, rho.data_ptr(), ux.data_ptr(), uy.data_ptr(), _stream_ptr(stream))
        return rho, ux, uy

    def residual(self, update_prev: bool = True, stream=None, raise_unstable: bool = True) -> np.ndarray:
        out = np.zeros((len(self.grids), _abi.LBM_NSTAT), dtype=np.float64)
        code = _abi.lib().lbm_residual(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       int(update_prev), _stream_ptr(stream))
        if code == _abi.LBM_ERR_UNSTABLE and not raise_unstable:
            return out
        _abi.check("lbm_residual", code)
        return out

    def step_residual(self, update_prev: bool = True, stream=None,
                      raise_unstable: bool = True) -> np.ndarray:
        """Statistics of the current level (as residual()) and one step, in one launch."""
        out = np.zeros((len(self.grids), _abi.LBM_NSTAT), dtype=np.float64)
        code = _abi.lib().lbm_step_residual(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            int(update_prev), _stream_ptr(stream))
        if code == _abi.LBM_ERR_UNSTABLE and not raise_unstable:
            return out
        _abi.check("lbm_step_residual", code)
        return out

    def set_persistent(self, on: bool = True) -> None:
        """step(n > 1) runs all n steps in one persistent launch (grid barrier between steps)."""
        call("lbm_set_persistent", self._h, int(bool(on)))

    def barrier_selftest(self, arrive_all: bool, limit_ms: float, stream=None) -> int:
        """Bounded grid-barrier self-test; returns the status code without raising."""
        status = torch.zeros(1, dtype=torch.int32, device=self.device)
        return int(_abi.lib().lbm_barrier_selftest(self._h, ctypes.c_void_p(status.data_ptr()),
                                                   int(bool(arrive_all)), float(limit_ms),
                                                   _stream_ptr(stream)))

    def stream_probe(self, variant: int, stream=None) -> None:
        """Replace the state by its streamed populations, through the step kernel's
        gather with tile shape `variant` (collision replaced by the identity)."""
        call("lbm_stream_probe", self._h, int(variant), _stream_ptr(stream))

    def reinit(self, rho: torch.Tensor, ux: torch.Tensor, uy: torch.Tensor, neq_mode: int = 1,
               stream=None) -> None:
        for t in (rho, ux, uy):
            assert t.dtype == torch.float32 and t.is_contiguous() and t.numel() == self.cells
        call("lbm_reinit_from_macro", self._h, rho.data_ptr(), ux.data_ptr(), uy.data_ptr(),
             int(neq_mode), _stream_ptr(stream))

    def vorticity(self, ux: torch.Tensor, uy: torch.Tensor, stream=None) -> torch.Tensor:
        """omega = d_x u_y - d_y u_x of dense velocity fields (library stencils)."""
        for t in (ux, uy):
            assert t.dtype == torch.float32 and t.is_contiguous() and t.numel() == self.cells
        out = torch.empty(self.cells, dtype=torch.float32, device=self.device)
        call("lbm_vorticity", self._h, ux.data_ptr(), uy.data_ptr(), out.data_ptr(),
             _stream_ptr(stream))
        return out

    def export_f(self, stream=None) -> torch.Tensor:
        out = torch.empty(9 * self.cells, dtype=torch.float32, device=self.device)
        call("lbm_export_f", self._h, out.data_ptr(), _stream_ptr(stream))
        return out

    def set_state(self, gstar: torch.Tensor, stream=None) -> None:
        assert gstar.dtype == torch.float32 and gstar.is_contiguous() and gstar.numel() == 9 * self.cells
        call("lbm_set_state", self._h, gstar.data_ptr(), _stream_ptr(stream))

    def get_state(self, stream=None) -> torch.Tensor:
        out = torch.empty(9 * self.cells, dtype=torch.float32, device=self.device)
        call("lbm_get_state", self._h, out.data_ptr(), _stream_ptr(stream))
        return out

    def autotune(self, reps: int = 10, stream=None):
        """Time every compiled step-kernel tile shape on this batch and keep the fastest.

        The state is unchanged.  Returns (chosen index, milliseconds per step per shape)."""
        ms = (ctypes.c_float * _abi.LBM_STEP_VARIANTS)()
        chosen = ctypes.c_int()
        call("lbm_autotune", self._h, int(reps), ms, ctypes.byref(chosen), _stream_ptr(stream))
        return chosen.value, list(ms)

    def set_step_variant(self, variant: int) -> None:
        call("lbm_set_step_variant", self._h, int(variant))

    def step_variant(self):
        """(index, rows per tile, stages, CTAs per SM) of the step kernel in use."""
        v = [ctypes.c_int() for _ in range(4)]
        call("lbm_get_step_variant", self._h, *[ctypes.byref(x) for x in v])
        return tuple(x.value for x in v)

    def steps_done(self) -> int:
        v = ctypes.c_longlong()
        call("lbm_steps_done", self._h, ctypes.byref(v))
        return v.value

    # ------------------------------------------------------------- adjoint
    def adjoint_macro(self, gstar: torch.Tensor, drho: torch.Tensor, dux: torch.Tensor,
                      duy: torch.Tensor, stream=None) -> torch.Tensor:
        """Adjoint seed mu_N of a loss on lbm_macro's outputs at the state gstar (canonical)."""
        for t in (drho, dux, duy):
            assert t.dtype == torch.float32 and t.is_contiguous() and t.numel() == self.cells
        assert gstar.dtype == torch.float32 and gstar.numel() == 9 * self.cells
        mu = torch.empty(9 * self.cells, dtype=torch.float32, device=self.device)
        call("lbm_adjoint_macro", self._h, gstar.data_ptr(), drho.data_ptr(), dux.data_ptr(),
             duy.data_ptr(), mu.data_ptr(), _stream_ptr(stream))
        return mu

    def adjoint_step(self, gstar_prev: torch.Tensor, mu: torch.Tensor, out=None,
                     stream=None) -> torch.Tensor:
        """mu_{n-1} from mu_n and the stored state s_{n-1} (canonical)."""
        assert gstar_prev.numel() == 9 * self.cells and mu.numel() == 9 * self.cells
        if out is None:
            out = torch.empty_like(mu)
        call("lbm_adjoint_step", self._h, gstar_prev.data_ptr(), mu.data_ptr(), out.data_ptr(),
             _stream_ptr(stream))
        return out

    def adjoint_reinit(self, mu: torch.Tensor, rho: torch.Tensor, ux: torch.Tensor,
                       uy: torch.Tensor, neq_mode: int = 1, stream=None):
        """(dL/drho, dL/dux, dL/duy) of the fields given to reinit, from mu_0."""
        for t in (rho, ux, uy):
            assert t.dtype == torch.float32 and t.is_contiguous() and t.numel() == self.cells
        scratch = torch.empty(3 * self.cells, dtype=torch.float32, device=self.device)
        out = [torch.empty(self.cells, dtype=torch.float32, device=self.device) for _ in range(3)]
        call("lbm_adjoint_reinit", self._h, mu.data_ptr(), rho.data_ptr(), ux.data_ptr(),
             uy.data_ptr(), int(neq_mode), scratch.data_ptr(), *[o.data_ptr() for o in out],
             _stream_ptr(stream))
        return tuple(out)

    def split(self, dense: torch.Tensor, per_cell: int = 1):
        """Split a dense (or canonical, per_cell=9) field into per-grid [.., ny, nx] views."""
        out = []
        for k, g in enumerate(self.grids):
            a, b = self.cell_offsets[k] * per_cell, self.cell_offsets[k + 1] * per_cell
            shape = (per_cell, g.ny, g.nx) if per_cell > 1 else (g.ny, g.nx)
            out.append(dense[a:b].view(*shape))
        return out

    def close(self) -> None:
        if self._h:
            _abi.lib().lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
