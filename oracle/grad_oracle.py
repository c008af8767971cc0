"""Differentiable FP64 reference of the hybrid pipeline, for reference gradients.

TEST INFRASTRUCTURE ONLY: used by the test suite to produce the FP64 reference
gradients that the CUDA adjoint kernels are compared with.  The product path never
imports it.

What it restates, in float64 torch CPU tensors so that torch's reverse-mode
autodiff (a library routine) yields exact gradients of the composite map:
  * the LBM of Sec. 2.1 in the oracle's own order (collision -> streaming with
    halfway bounce-back -> Zou-He completion), with Guo forcing, the moments with
    the half-force correction, and the re-initialisation from macroscopic fields
    of the hybrid framework (Sec. 2.3: f = f^eq + f^neq, the Chapman-Enskog estimate
    f^neq_i = -(tau w_i rho / c_s^2) Q_iab d_a u_b with central differences, one-sided
    next to solid cells and open ends);
  * the FNO forward pass of Sec. 2.2 (truncated DFT over the kept modes, per-mode
    complex channel mixing, Hermitian-half inverse, 1x1 layer, activation after every
    layer, coordinate channels, decoder) with explicit DFT matrices;
  * the training objective of the differentiable hybrid step: the mean squared error
    of (rho, u_x, u_y) over fluid cells after n LBM steps that follow the
    re-initialisation from given (or FNO-predicted) fields.

Every forward here is pinned to the C / numpy oracle value for value (to FP64
round-off), and every gradient to central finite differences, by the tests in
`tests/test_grad_oracle.py`.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np
import torch

from . import Grid, lattice
from .fno_oracle import bf16, coordinate_channels, kept_ky

BC_PERIODIC, BC_PRESSURE, BC_VELOCITY = 0, 1, 2
_T = torch.float64


class TorchLattice:
    """One lattice (grid + solid mask) with its streaming gather map precomputed."""

    def __init__(self, grid: Grid, solid: np.ndarray):
        self.g = grid
        self.solid_np = np.asarray(solid, dtype=bool)
        ny, nx = self.solid_np.shape
        assert (ny, nx) == (grid.ny, grid.nx)
        self.ny, self.nx, self.N = ny, nx, nx * ny
        cx, cy, w, opp = lattice()
        self.cx = torch.tensor(cx, dtype=_T)[:, None, None]
        self.cy = torch.tensor(cy, dtype=_T)[:, None, None]
        self.w = torch.tensor(w, dtype=_T)[:, None, None]
        self.cxi, self.cyi, self.opp = cx, cy, opp
        self.solid = torch.from_numpy(self.solid_np)
        self.fluid = ~self.solid
        self.periodic_x = grid.bc_west == BC_PERIODIC
        # pull map: population i of cell (x, y) reads fstar_i(x - c_i) if that is a fluid
        # cell of the domain, fstar_opp(i)(x) if it is solid; solid cells keep their own
        # values; populations entering through an open end read a zero placeholder (slot
        # 9 N) that the Zou-He completion overwrites
        Y, X = np.mgrid[0:ny, 0:nx]
        idx = np.empty((9, ny, nx), dtype=np.int64)
        for i in range(9):
            xs = X - cx[i]
            ys = (Y - cy[i]) % ny
            out = (xs < 0) | (xs >= nx)
            if self.periodic_x:
                xs = xs % nx
                out = np.zeros_like(out)
            xs_c = np.clip(xs, 0, nx - 1)
            src_solid = self.solid_np[ys, xs_c]
            own = i * self.N + Y * nx + X
            idx[i] = np.where(self.solid_np, own,
                              np.where(out, 9 * self.N,
                                       np.where(src_solid, opp[i] * self.N + Y * nx + X,
                                                i * self.N + ys * nx + xs_c)))
        self.pull_idx = torch.from_numpy(idx.reshape(-1))

    # -------------------------------------------------------------- LBM pieces
    def moments(self, f: torch.Tensor):
        g = self.g
        rho = f.sum(0)
        ux = ((self.cx * f).sum(0) + 0.5 * g.fx) / rho
        uy = ((self.cy * f).sum(0) + 0.5 * g.fy) / rho
        return rho, ux, uy

    def equilibrium(self, rho, ux, uy):
        cu = self.cx * ux + self.cy * uy
        uu = ux * ux + uy * uy
        return self.w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)

    def collide(self, f: torch.Tensor) -> torch.Tensor:
        """BGK relaxation with the Guo source on fluid cells; solid cells unchanged."""
        g = self.g
        rho, ux, uy = self.moments(f)
        feq = self.equilibrium(rho, ux, uy)
        cu = self.cx * ux + self.cy * uy
        sx = 3.0 * (self.cx - ux) + 9.0 * cu * self.cx
        sy = 3.0 * (self.cy - uy) + 9.0 * cu * self.cy
        src = (1.0 - 0.5 / g.tau) * self.w * (sx * g.fx + sy * g.fy)
        fs = f - (f - feq) / g.tau + src
        return torch.where(self.solid, f, fs)

    def boundary(self, f: torch.Tensor) -> torch.Tensor:
        """Zou-He completion on the fluid cells of the open end columns."""
        g = self.g
        if g.bc_west != BC_PERIODIC:
            col = self._zou_he(f[:, :, 0], west=True, kind=g.bc_west, value=g.west_value,
                               fluid=self.fluid[:, 0])
            f = torch.cat([col[:, :, None], f[:, :, 1:]], dim=2)
        if g.bc_east != BC_PERIODIC:
            col = self._zou_he(f[:, :, -1], west=False, kind=g.bc_east, value=g.east_value,
                               fluid=self.fluid[:, -1])
            f = torch.cat([f[:, :, :-1], col[:, :, None]], dim=2)
        return f

    @staticmethod
    def _zou_he(col, west, kind, value, fluid):
        r = [col[i] for i in range(9)]
        if west:
            known = r[0] + r[2] + r[4] + 2.0 * (r[3] + r[6] + r[7])
            if kind == BC_PRESSURE:
                rho = torch.full_like(known, value)
                ux = 1.0 - known / rho
            else:
                ux = torch.full_like(known, value)
                rho = known / (1.0 - ux)
            ru = rho * ux
            new = {1: r[3] + (2.0 / 3.0) * ru,
                   5: r[7] - 0.5 * (r[2] - r[4]) + ru / 6.0,
                   8: r[6] + 0.5 * (r[2] - r[4]) + ru / 6.0}
        else:
            known = r[0] + r[2] + r[4] + 2.0 * (r[1] + r[5] + r[8])
            if kind == BC_PRESSURE:
                rho = torch.full_like(known, value)
                ux = -1.0 + known / rho
            else:
                ux = torch.full_like(known, value)
                rho = known / (1.0 + ux)
            ru = rho * ux
            new = {3: r[1] - (2.0 / 3.0) * ru,
                   7: r[5] + 0.5 * (r[2] - r[4]) - ru / 6.0,
                   6: r[8] - 0.5 * (r[2] - r[4]) - ru / 6.0}
        for i, v in new.items():
            r[i] = torch.where(fluid, v, r[i])
        return torch.stack(r)

    def stream(self, fstar: torch.Tensor) -> torch.Tensor:
        ext = torch.cat([fstar.reshape(-1), fstar.new_zeros(1)])
        f = ext[self.pull_idx].reshape(9, self.ny, self.nx)
        return self.boundary(f)

    def step(self, f: torch.Tensor) -> torch.Tensor:
        return self.stream(self.collide(f))

    def macro(self, f: torch.Tensor):
        rho, ux, uy = self.moments(f)
        one = torch.ones_like(rho)
        zero = torch.zeros_like(rho)
        return (torch.where(self.solid, one, rho), torch.where(self.solid, zero, ux),
                torch.where(self.solid, zero, uy))

    def _deriv(self, v: torch.Tensor, axis: int) -> torch.Tensor:
        """Central difference where both neighbours along `axis` are fluid cells of the
        domain, one-sided where one is, zero where none is (y always periodic)."""
        dim = 1 if axis == 0 else 0
        vp = torch.roll(v, -1, dims=dim)  # value at the + neighbour
        vm = torch.roll(v, 1, dims=dim)
        fp = torch.roll(self.fluid, -1, dims=dim)
        fm = torch.roll(self.fluid, 1, dims=dim)
        if axis == 0 and not self.periodic_x:
            fp = fp.clone()
            fm = fm.clone()
            fp[:, -1] = False
            fm[:, 0] = False
        return torch.where(fp & fm, 0.5 * (vp - vm),
                           torch.where(fp, vp - v, torch.where(fm, v - vm, torch.zeros_like(v))))

    def reinit(self, rho, ux, uy, neq_mode: int = 1) -> torch.Tensor:
        """f^eq(rho, u) + f^neq on fluid cells, w_i on solid cells, then Zou-He."""
        feq = self.equilibrium(rho, ux, uy)
        f = feq
        if neq_mode:
            d = {(0, 0): self._deriv(ux, 0), (0, 1): self._deriv(uy, 0),
                 (1, 0): self._deriv(ux, 1), (1, 1): self._deriv(uy, 1)}
            c = (self.cx, self.cy)
            qd = 0.0
            for a in range(2):
                for b in range(2):
                    qd = qd + (c[a] * c[b] - (1.0 / 3.0 if a == b else 0.0)) * d[(a, b)]
            f = feq - (self.g.tau * self.w * rho * 3.0) * qd
        f = torch.where(self.solid, self.w.expand(9, self.ny, self.nx), f)
        return self.boundary(f)

    def run(self, f: torch.Tensor, nsteps: int) -> torch.Tensor:
        for _ in range(nsteps):
            f = self.step(f)
        return f

    # ---------------------------------------------------------- training loss
    def loss_after_steps(self, rho0, ux0, uy0, nsteps: int, target, neq_mode: int = 1):
        """MSE over fluid cells of (rho, u_x, u_y) after nsteps LBM steps that follow the
        re-initialisation from (rho0, ux0, uy0); target = (rho*, ux*, uy*)."""
        f = self.run(self.reinit(rho0, ux0, uy0, neq_mode), nsteps)
        rho, ux, uy = self.macro(f)
        fl = self.fluid
        n = 3.0 * float(fl.sum())
        return (((rho - target[0])[fl] ** 2).sum() + ((ux - target[1])[fl] ** 2).sum() +
                ((uy - target[2])[fl] ** 2).sum()) / n


# ------------------------------------------------------------------- FNO
def _gelu(x):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def _dft_mats(H: int, W: int, m: int):
    """Forward factors Fy [2m, H], Fx [W, m] and inverse Gy [H, 2m], Gx [m, W] (complex128),
    phases reduced (k n mod N) before scaling."""
    ky = kept_ky(H, m)
    kx = np.arange(m)

    def tw(k, n, N, sign):
        ph = np.mod(np.outer(k, n), N).astype(np.float64)
        return torch.from_numpy(np.exp(1j * sign * 2.0 * math.pi * ph / N))

    ckx = torch.from_numpy(np.where(kx == 0, 1.0, 2.0)).to(torch.complex128)
    return (tw(ky, np.arange(H), H, -1.0), tw(np.arange(W), kx, W, -1.0),
            tw(np.arange(H), ky, H, +1.0), ckx[:, None] * tw(kx, np.arange(W), W, +1.0))


def fno_forward(shape, params: Dict[str, torch.Tensor], phi: torch.Tensor,
                activation: str = "gelu") -> torch.Tensor:
    """FNO forward on phi [B, c_in, H, W] (float64 tensors; parameters already rounded to
    bfloat16 by the caller, see `bf16_params`)."""
    act = _gelu if activation == "gelu" else torch.relu
    B, _, H, W = phi.shape
    coords = torch.from_numpy(coordinate_channels(H, W))[None].expand(B, 2, H, W)
    x = torch.cat([phi, coords], dim=1)

    def pw(w, b, t):
        return torch.einsum("oi,bihw->bohw", w, t) + b[None, :, None, None]

    h = act(pw(params["lift0.w"], params["lift0.b"], x))
    theta = pw(params["lift1.w"], params["lift1.b"], h)
    pad = getattr(shape, "padding", 0)
    if pad:  # zero padding of the latent field, cropped after the last layer
        theta = torch.nn.functional.pad(theta, (0, pad, 0, pad))
    Hp, Wp = H + pad, W + pad
    Fy, Fx, Gy, Gx = _dft_mats(Hp, Wp, shape.modes)
    for n in range(shape.layers):
        R = torch.cat([torch.complex(params[f"layer{n}.r1.re"], params[f"layer{n}.r1.im"]),
                       torch.complex(params[f"layer{n}.r2.re"], params[f"layer{n}.r2.im"])],
                      dim=2)
        X = Fy @ theta.to(torch.complex128) @ Fx
        Yh = torch.einsum("bikl,iokl->bokl", X, R)
        s = torch.real(Gy @ Yh @ Gx) / (Hp * Wp)
        theta = act(pw(params[f"layer{n}.w"], params[f"layer{n}.b"], theta) + s)
    h = theta[:, :, :H, :W]
    for l in range(shape.dec_layers):
        h = act(pw(params[f"dec{l}.w"], params[f"dec{l}.b"], h))
    return pw(params["out.w"], params["out.b"], h)


def bf16_params(params: Dict[str, np.ndarray], requires_grad: bool = False):
    """bfloat16-rounded copies of the parameters as float64 leaf tensors."""
    return {k: torch.tensor(bf16(v), dtype=_T, requires_grad=requires_grad)
            for k, v in params.items()}


def hybrid_loss(lat: TorchLattice, shape, params, phi, nsteps: int, target,
                neq_mode: int = 1, activation: str = "gelu"):
    """Differentiable hybrid training objective for one grid: the FNO predicts
    (delta rho, u_x, u_y) from phi [1, c_in, H, W], the populations are re-initialised
    from (1 + delta rho, u), nsteps LBM steps follow, and the loss is the MSE of the
    final (rho, u) against the target over fluid cells."""
    y = fno_forward(shape, params, phi, activation)[0]
    return lat.loss_after_steps(1.0 + y[0], y[1], y[2], nsteps, target, neq_mode)
