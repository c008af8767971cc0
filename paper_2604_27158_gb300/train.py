"""Differentiable hybrid training step: FNO prediction -> re-initialisation -> LBM steps -> loss.

The FNO forward/backward run in the library's training kernels (fno_train_forward /
fno_train_backward: FP32 master parameters, saved activations, the spectral layer's
adjoint), the LBM part in its adjoint kernels (adjoint.LbmRollout).  torch.autograd
chains them; the loss (MSE of rho, u over fluid cells) and the optimiser update are
the caller's torch code.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from ._abi import call, fno_train_sizes
from .adjoint import fluid_mse, lbm_rollout
from .fno import FnoShape
from .lbm import Lattice, _stream_ptr


def fno_train_query(shape: FnoShape, B: int, H: int, W: int) -> fno_train_sizes:
    out = fno_train_sizes()
    cfg = shape.c()
    call("fno_train_query", ctypes.byref(cfg), int(B), int(H), int(W), ctypes.byref(out))
    return out


class _Buffers:
    """Saved-activation and scratch buffers per (B, H, W), reused across steps."""

    def __init__(self):
        self.cache = {}

    def get(self, shape: FnoShape, B, H, W, device):
        key = (shape, B, H, W)
        if key not in self.cache:
            sz = fno_train_query(shape, B, H, W)
            saved = torch.empty(sz.saved_bytes // 4, dtype=torch.float32, device=device)
            ws = torch.empty(sz.ws_bytes + 256, dtype=torch.uint8, device=device)
            off = (-ws.data_ptr()) % 256
            self.cache[key] = (saved, ws[off:off + sz.ws_bytes])
        return self.cache[key]


_BUFFERS = _Buffers()


class FnoTrainFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, x: torch.Tensor, shape: FnoShape):
        assert params.dtype == torch.float32 and x.dtype == torch.float32 and x.dim() == 4
        params = params.detach().contiguous()
        x = x.detach().contiguous()
        B, cin, H, W = x.shape
        assert cin == shape.c_in
        saved, ws = _BUFFERS.get(shape, B, H, W, x.device)
        out = torch.empty((B, shape.c_out, H, W), dtype=torch.float32, device=x.device)
        cfg = shape.c()
        call("fno_train_forward", ctypes.byref(cfg), params.data_ptr(), x.data_ptr(),
             out.data_ptr(), B, H, W, saved.data_ptr(), ws.data_ptr(), _stream_ptr(None))
        ctx.shape, ctx.dims = shape, (B, H, W)
        ctx.need_x = ctx.needs_input_grad[1]
        ctx.save_for_backward(params)
        ctx.saved_buf, ctx.ws = saved, ws
        return out

    @staticmethod
    def backward(ctx, dout):
        (params,) = ctx.saved_tensors
        B, H, W = ctx.dims
        shape = ctx.shape
        dparams = torch.empty_like(params)
        dx = (torch.empty((B, shape.c_in, H, W), dtype=torch.float32, device=params.device)
              if ctx.need_x else None)
        cfg = shape.c()
        call("fno_train_backward", ctypes.byref(cfg), params.data_ptr(),
             dout.float().contiguous().data_ptr(), ctx.saved_buf.data_ptr(), dparams.data_ptr(),
             dx.data_ptr() if dx is not None else None, B, H, W, ctx.ws.data_ptr(),
             _stream_ptr(None))
        return dparams, dx, None


def fno_apply(shape: FnoShape, params: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """FNO(x) with FP32 parameters, differentiable in params and x (training kernels)."""
    return FnoTrainFn.apply(params, x, shape)


def hybrid_loss(lat: Lattice, shape: FnoShape, params: torch.Tensor, x: torch.Tensor,
                nsteps: int, target: Sequence[torch.Tensor], every: int = 8,
                neq_mode: int = 1, fluid: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Training objective of the differentiable hybrid step for a batch of B equal grids:
    the FNO predicts (delta rho, u_x, u_y) from x [B, c_in, H, W]; the lattice is
    re-initialised from (1 + delta rho, u) and advanced nsteps steps; the loss is the MSE
    of the final (rho, u) against `target` (dense fields) over fluid cells.  No clamping
    of the prediction (the inference driver clamps; here gradients must flow)."""
    y = fno_apply(shape, params, x)
    rho0 = (1.0 + y[:, 0]).reshape(-1)
    ux0 = y[:, 1].reshape(-1)
    uy0 = y[:, 2].reshape(-1)
    out = lbm_rollout(lat, rho0, ux0, uy0, nsteps, every=every, neq_mode=neq_mode)
    return fluid_mse(lat, out, target, fluid)
