"""Differentiable LBM rollout: reinit -> n fused steps -> moments as a torch.autograd.Function.

Forward runs the library's reinit, step and macro kernels, keeping the stored state
every `every` steps (checkpoints).  Backward runs the adjoint kernels of the library
(lbm_adjoint_macro / lbm_adjoint_step / lbm_adjoint_reinit), recomputing the states
between two checkpoints with the forward step kernel.  Memory: one canonical state
(36 B per cell) per checkpoint plus `every` states for the segment being reversed.

The Lattice's state after backward is the last recomputed state, not the state after
the forward pass: a caller that continues stepping must set it again.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from .lbm import Lattice


class LbmRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, ux0, uy0, lat: Lattice, nsteps: int, every: int, neq_mode: int):
        assert nsteps >= 0 and every >= 1
        fields = [t.detach().float().contiguous() for t in (rho0, ux0, uy0)]
        lat.reinit(*fields, neq_mode=neq_mode)
        checkpoints = []
        done = 0
        while done < nsteps:
            checkpoints.append(lat.get_state())
            k = min(every, nsteps - done)
            lat.step(k)
            done += k
        final = lat.get_state()
        rho, ux, uy = lat.macro()
        ctx.lat, ctx.nsteps, ctx.every, ctx.neq_mode = lat, nsteps, every, neq_mode
        ctx.checkpoints, ctx.final = checkpoints, final
        ctx.save_for_backward(*fields)
        return rho, ux, uy

    @staticmethod
    def backward(ctx, drho, dux, duy):
        lat: Lattice = ctx.lat
        rho0, ux0, uy0 = ctx.saved_tensors
        g = [torch.zeros(lat.cells, dtype=torch.float32, device=lat.device) if t is None
             else t.float().contiguous() for t in (drho, dux, duy)]
        mu = lat.adjoint_macro(ctx.final, *g)
        spare = torch.empty_like(mu)
        for seg in reversed(range(len(ctx.checkpoints))):
            k = min(ctx.every, ctx.nsteps - seg * ctx.every)
            states = [ctx.checkpoints[seg]]
            if k > 1:
                lat.set_state(ctx.checkpoints[seg])
                for _ in range(k - 1):
                    lat.step(1)
                    states.append(lat.get_state())
            for j in reversed(range(k)):
                lat.adjoint_step(states[j], mu, out=spare)
                mu, spare = spare, mu
        d = lat.adjoint_reinit(mu, rho0, ux0, uy0, ctx.neq_mode)
        return d[0], d[1], d[2], None, None, None, None


def lbm_rollout(lat: Lattice, rho0: torch.Tensor, ux0: torch.Tensor, uy0: torch.Tensor,
                nsteps: int, every: int = 8, neq_mode: int = 1):
    """(rho, u_x, u_y) after re-initialising `lat` from (rho0, ux0, uy0) and nsteps steps;
    differentiable with respect to the three dense input fields."""
    return LbmRollout.apply(rho0, ux0, uy0, lat, int(nsteps), int(every), int(neq_mode))


def fluid_mse(lat: Lattice, fields, target, fluid: Optional[torch.Tensor] = None):
    """Mean over fluid cells and the three fields of the squared difference."""
    if fluid is None:
        fluid = ~torch.from_numpy(np.concatenate([s.ravel() for s in lat.solid])).to(lat.device)
    n = 3.0 * float(fluid.sum())
    return sum(((a - b)[fluid] ** 2).sum() for a, b in zip(fields, target)) / n
