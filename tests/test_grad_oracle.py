"""Pins of the differentiable FP64 reference (oracle/grad_oracle.py).

Its forwards must equal the C / numpy oracle (to FP64 round-off), and its gradients
must equal central finite differences (eps = 1e-3, FP64) of the same forward: the
training objective of the differentiable hybrid step (MSE of rho, u after LBM steps
that follow the re-initialisation, Sec. 2.3) with respect to the initial fields and
to the FNO parameters (Sec. 2.2).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import fno_oracle as fo
from oracle import grad_oracle as go

T = torch.float64


def _cases():
    out = []
    s, _, _ = synth.porous_media(40, 24, 3, 4, seed=2)
    out.append(("porous pressure", oracle.Grid(nx=40, ny=24, tau=0.7, bc_west=1, bc_east=1,
                                               west_value=1.01, east_value=1.0), s))
    s, _ = synth.flow_past_disks(48, 24, seed=3, rmax=4)
    out.append(("disks velocity", oracle.Grid(nx=48, ny=24, tau=0.6, bc_west=2, bc_east=1,
                                              west_value=0.04, east_value=1.0), s))
    s, _ = synth.channel_with_disks(32, 20, 2, 2, 3, seed=1)
    out.append(("forced channel", oracle.Grid(nx=32, ny=20, tau=0.8, fx=1e-4, fy=2e-5), s))
    return out


def _fields(ny, nx, seed):
    sf = synth.smooth_macro_fields(nx, ny, seed=seed, drho=1e-2, umax=0.05)
    return [np.asarray(a, dtype=np.float64) for a in sf]


@pytest.mark.parametrize("k", range(3))
def test_torch_lbm_equals_c_oracle(k):
    name, g, solid = _cases()[k]
    lat = go.TorchLattice(g, solid)
    rho, ux, uy = _fields(g.ny, g.nx, seed=k)
    for neq in (0, 1):
        f_c = oracle.reinit(g, solid, rho, ux, uy, neq_mode=neq)
        f_t = lat.reinit(*(torch.from_numpy(a) for a in (rho, ux, uy)), neq_mode=neq)
        np.testing.assert_allclose(f_t.numpy(), f_c, rtol=0, atol=1e-15)
    f_c = oracle.run(g, solid, f_c, 25)
    f_t = lat.run(f_t, 25)
    np.testing.assert_allclose(f_t.numpy(), f_c, rtol=0, atol=1e-14)
    for a, b in zip(lat.macro(f_t), oracle.macro(g, solid, f_c)):
        np.testing.assert_allclose(a.numpy(), b, rtol=0, atol=1e-14)


def test_torch_fno_equals_numpy_oracle():
    shape = synth.FnoShape(width=8, layers=2, modes=3, dec_size=8)
    params = synth.fno_random_params(shape, seed=4, out_scale=1.0)
    x = fo.bf16(np.random.default_rng(0).standard_normal((2, 4, 12, 16)))
    ref = fo.fno_forward(shape, params, x)
    got = go.fno_forward(shape, go.bf16_params(params), torch.from_numpy(x)).numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def _central(fn, xs, ds, eps):
    with torch.no_grad():
        lp = fn([x + eps * d for x, d in zip(xs, ds)])
        lm = fn([x - eps * d for x, d in zip(xs, ds)])
    return float((lp - lm) / (2.0 * eps))


def _central_directional(fn, xs, ds, eps):
    """Central differences at eps and eps/2 combined by Richardson extrapolation: the
    O(eps^2) truncation term of the central difference cancels (plain central differences
    at eps = 1e-3 carry a relative error of ~1e-4 on these objectives)."""
    return (4.0 * _central(fn, xs, ds, 0.5 * eps) - _central(fn, xs, ds, eps)) / 3.0


def test_loss_gradient_wrt_fields_matches_finite_differences():
    """32 x 32 porous medium, pressure inlet/outlet, 8 LBM steps after the reinit."""
    solid, _, _ = synth.porous_media(32, 32, 3, 4, seed=5)
    g = oracle.Grid(nx=32, ny=32, tau=0.7, bc_west=1, bc_east=1, west_value=1.01,
                    east_value=1.0)
    lat = go.TorchLattice(g, solid)
    rho, ux, uy = (torch.from_numpy(a) for a in _fields(32, 32, seed=9))
    tgt = tuple(torch.from_numpy(a) for a in _fields(32, 32, seed=10))
    xs = [t.clone().requires_grad_(True) for t in (rho, ux, uy)]
    fn = lambda v: lat.loss_after_steps(v[0], v[1], v[2], 8, tgt)
    loss = fn(xs)
    grads = torch.autograd.grad(loss, xs)
    rng = np.random.default_rng(1)
    for _ in range(4):
        ds = [torch.from_numpy(rng.standard_normal((32, 32))) for _ in range(3)]
        fd = _central_directional(fn, [x.detach() for x in xs], ds, 1e-3)
        ad = float(sum((gr * d).sum() for gr, d in zip(grads, ds)))
        assert abs(fd - ad) <= 1e-8 * abs(ad), (fd, ad)


def test_loss_gradient_every_component_on_a_tiny_grid():
    """Every input component of a 10 x 8 grid with a velocity inlet and one solid block."""
    solid = np.zeros((8, 10), dtype=bool)
    solid[3:5, 4:6] = True
    g = oracle.Grid(nx=10, ny=8, tau=0.65, bc_west=2, bc_east=1, west_value=0.03,
                    east_value=1.0)
    lat = go.TorchLattice(g, solid)
    rho, ux, uy = (torch.from_numpy(a) for a in _fields(8, 10, seed=3))
    tgt = tuple(torch.from_numpy(a) for a in _fields(8, 10, seed=4))
    xs = [t.clone().requires_grad_(True) for t in (rho, ux, uy)]
    fn = lambda v: lat.loss_after_steps(v[0], v[1], v[2], 5, tgt)
    grads = [gr.numpy() for gr in torch.autograd.grad(fn(xs), xs)]
    base = [x.detach() for x in xs]
    eps = 1e-3
    for c in range(3):
        fd = np.zeros((8, 10))
        for y in range(8):
            for x in range(10):
                d = [torch.zeros(8, 10, dtype=T) for _ in range(3)]
                d[c][y, x] = 1.0
                fd[y, x] = _central_directional(fn, base, d, eps)
        np.testing.assert_allclose(grads[c], fd, rtol=1e-7, atol=1e-13)
        assert np.all(grads[c][solid] == 0.0)  # solid cells do not enter the loss


def test_hybrid_loss_gradient_wrt_fno_parameters_matches_finite_differences():
    shape = synth.FnoShape(width=8, layers=2, modes=3, dec_size=8)
    params = synth.fno_random_params(shape, seed=2, out_scale=1e-1)
    solid, _, _ = synth.porous_media(24, 16, 2, 3, seed=6)
    g = oracle.Grid(nx=24, ny=16, tau=0.7, bc_west=1, bc_east=1, west_value=1.01,
                    east_value=1.0)
    lat = go.TorchLattice(g, solid)
    phi = torch.from_numpy(fo.bf16(np.stack([np.zeros((16, 24)), np.zeros((16, 24)),
                                             np.zeros((16, 24)), solid.astype(float)])[None]))
    tgt = tuple(torch.from_numpy(a) for a in _fields(16, 24, seed=7))
    P = go.bf16_params(params, requires_grad=True)
    names = list(P)
    fn = lambda v: go.hybrid_loss(lat, shape, dict(zip(names, v)), phi, 6, tgt)
    grads = torch.autograd.grad(fn([P[k] for k in names]), [P[k] for k in names])
    rng = np.random.default_rng(5)
    for _ in range(3):
        ds = [torch.from_numpy(rng.standard_normal(P[k].shape)) for k in names]
        fd = _central_directional(fn, [P[k].detach() for k in names], ds, 1e-3)
        ad = float(sum((gr * d).sum() for gr, d in zip(grads, ds)))
        assert abs(fd - ad) <= 1e-7 * abs(ad), (fd, ad)
