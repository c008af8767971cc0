"""Training the initialisation FNO of the steady framework (Sec. 2.3, Fig. 3a) on LBM data.

The paper trains its FNOs offline on LBM snapshots of converged porous-media flows and then
uses the prediction as the initial state of the LBM.  This module does the same with this
library's kernels only: the training data are steady (long-run) states of the fused LBM
step, and the network is fitted with the FNO training kernels (fno_train_forward /
fno_train_backward); torch supplies the optimiser update and the loss reduction.

Targets are normalised per channel by their standard deviation over fluid cells while
training; the scale is folded into the output layer afterwards, so the returned parameters
predict absolute (rho - 1, u_x, u_y) and plug into the inference path (fno_forward) and the
hybrid driver unchanged.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np
import torch

from .fno import FnoShape
from .lbm import GridSpec, Lattice
from .train import fno_apply


def steady_states(grid: GridSpec, masks: Sequence[np.ndarray], steps: int, batch: int = 64,
                  device: str = "cuda") -> torch.Tensor:
    """(rho - 1, u_x, u_y) [N, 3, ny, nx] after `steps` fused LBM steps from rest, for each
    mask (batches of `batch` grids per launch)."""
    out: List[torch.Tensor] = []
    for i in range(0, len(masks), batch):
        mk = list(masks[i:i + batch])
        lat = Lattice([grid] * len(mk), mk, device=device)
        lat.autotune(reps=3)
        lat.step(int(steps))
        rho, ux, uy = lat.macro()
        B = len(mk)
        out.append(torch.stack([(rho - 1.0).view(B, grid.ny, grid.nx), ux.view(B, grid.ny, grid.nx),
                                uy.view(B, grid.ny, grid.nx)], dim=1))
        lat.close()
    return torch.cat(out)


def fno_inputs(masks: Sequence[np.ndarray], c_in: int = 4, device: str = "cuda") -> torch.Tensor:
    """FNO input of the steady framework: the default fields (rho - 1 = u = 0) and the mask,
    [N, 4, ny, nx] (or the mask alone for c_in = 1)."""
    m = torch.from_numpy(np.stack(masks).astype(np.float32)).to(device)
    if c_in == 1:
        return m[:, None].contiguous()
    x = torch.zeros((m.shape[0], 4, m.shape[1], m.shape[2]), device=device)
    x[:, 3] = m
    return x


def train_supervised(shape: FnoShape, params0: np.ndarray, x: torch.Tensor, y: torch.Tensor,
                     fluid: torch.Tensor, steps: int, batch: int = 8, lr: float = 2e-3,
                     seed: int = 0, log_every: int = 0) -> Tuple[np.ndarray, List[float]]:
    """Fit the FNO to y [N, c_out, H, W] from x [N, c_in, H, W] by Adam on the per-channel
    normalised MSE over fluid cells (`fluid` [N, H, W] bool), cosine learning-rate decay.

    Returns (FP32 parameters predicting absolute values, loss history)."""
    scale = torch.stack([y[:, c][fluid].std() for c in range(y.shape[1])]).clamp_min(1e-12)
    yn = y / scale[None, :, None, None]
    params = torch.nn.Parameter(torch.from_numpy(np.asarray(params0, np.float32)).to(x.device))
    opt = torch.optim.Adam([params], lr=lr)
    sched = torch.optim.lr_scheduler.LambdaLR(
        opt, lambda s: 0.5 * (1.0 + math.cos(math.pi * min(s, steps) / max(steps, 1))))
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    hist: List[float] = []
    for it in range(int(steps)):
        idx = torch.from_numpy(rng.choice(n, min(batch, n), replace=False)).to(x.device)
        pred = fno_apply(shape, params, x[idx])
        f = fluid[idx][:, None].expand(-1, y.shape[1], -1, -1)
        loss = ((pred - yn[idx]) ** 2)[f].mean()
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append(float(loss.detach()))
    # fold the normalisation into the output layer: out.w [c_out][S] and out.b [c_out] are
    # the last entries of the parameter pack
    p = params.detach().clone()
    co, S = shape.c_out, shape.dec_size
    nw = co * S
    w = p[-(nw + co):-co].view(co, S) * scale[:, None]
    b = p[-co:] * scale
    p[-(nw + co):-co] = w.reshape(-1)
    p[-co:] = b
    return p.cpu().numpy(), hist
