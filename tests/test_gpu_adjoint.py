"""GPU adjoint of the LBM part of the hybrid pipeline against FP64 reference gradients.

The loss is the training objective of the differentiable hybrid step: the MSE over
fluid cells of (rho, u_x, u_y) after n LBM steps that follow the re-initialisation
from (rho0, u0) (Sec. 2.3).  The CUDA path differentiates it with the library's
adjoint kernels behind torch.autograd (checkpoints every K steps, recomputation in
between); the reference is torch autograd through the FP64 restatement in
oracle/grad_oracle.py, itself pinned to the C oracle and to central finite
differences.  Bar: 1e-4 relative L2 per gradient field (FP32 adjoint of an FP32
forward against FP64).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import grad_oracle as go

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300.adjoint import lbm_rollout  # noqa: E402
from paper_2604_27158_gb300.lbm import GridSpec, Lattice  # noqa: E402

REL_GRAD = 1e-4


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_oracle(g):
    return oracle.Grid(nx=g.nx, ny=g.ny, tau=g.tau, fx=g.fx, fy=g.fy, bc_west=g.bc_west,
                       bc_east=g.bc_east, west_value=g.west_value, east_value=g.east_value)


def _fields(g, seed, drho=1e-2, umax=0.05):
    return [np.asarray(a, dtype=np.float32)
            for a in synth.smooth_macro_fields(g.nx, g.ny, seed=seed, drho=drho, umax=umax)]


def _batch():
    specs = []
    s, _, _ = synth.porous_media(32, 32, 3, 4, seed=5)
    specs.append((GridSpec(32, 32, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                           west_value=1.01, east_value=1.0), s))
    s, _ = synth.flow_past_disks(48, 24, seed=3, rmax=4)
    specs.append((GridSpec(48, 24, 0.6, bc_west=P.BC_VELOCITY, bc_east=P.BC_PRESSURE,
                           west_value=0.04, east_value=1.0), s))
    s, _ = synth.channel_with_disks(40, 20, 2, 2, 3, seed=1)
    specs.append((GridSpec(40, 20, 0.8, fx=1e-4, fy=2e-5), s))
    s = np.zeros((16, 33), dtype=bool)  # no solid cells, ragged width
    specs.append((GridSpec(33, 16, 0.9), s))
    return specs


def _gpu_and_reference(specs, nsteps, every, neq_mode):
    lat = Lattice([g for g, _ in specs], [s for _, s in specs])
    offs = lat.cell_offsets
    ins = [[], [], []]
    tgts = [[], [], []]
    for k, (g, _) in enumerate(specs):
        a = _fields(g, seed=20 + k)
        t = _fields(g, seed=40 + k)
        for c in range(3):
            ins[c].append(a[c].ravel())
            tgts[c].append(t[c].ravel())
    x = [torch.from_numpy(np.concatenate(v)).cuda().requires_grad_(True) for v in ins]
    tgt = [torch.from_numpy(np.concatenate(v)).cuda() for v in tgts]
    out = lbm_rollout(lat, x[0], x[1], x[2], nsteps, every=every, neq_mode=neq_mode)
    loss = 0.0
    for k, (g, s) in enumerate(specs):
        fl = torch.from_numpy(~s.ravel()).cuda()
        n = 3.0 * float(fl.sum())
        sl = slice(offs[k], offs[k + 1])
        loss = loss + sum(((o[sl] - t[sl])[fl] ** 2).sum() for o, t in zip(out, tgt)) / n
    loss.backward()
    grads = [t.grad.detach().cpu().numpy() for t in x]
    results = []
    for k, (g, s) in enumerate(specs):
        sl = slice(offs[k], offs[k + 1])
        tl = go.TorchLattice(to_oracle(g), s)
        xr = [torch.from_numpy(ins[c][k].astype(np.float64).reshape(g.ny, g.nx)).requires_grad_(True)
              for c in range(3)]
        tr = tuple(torch.from_numpy(tgts[c][k].astype(np.float64).reshape(g.ny, g.nx))
                   for c in range(3))
        lr = tl.loss_after_steps(xr[0], xr[1], xr[2], nsteps, tr, neq_mode)
        ref = [v.numpy() for v in torch.autograd.grad(lr, xr)]
        got = [grads[c][sl].reshape(g.ny, g.nx) for c in range(3)]
        results.append((g, s, got, ref))
    lat.close()
    return results


def _check(results, label):
    for g, s, got, ref in results:
        for c, name in enumerate(("rho", "ux", "uy")):
            err = np.linalg.norm(got[c] - ref[c]) / np.linalg.norm(ref[c])
            print(f"{label} {g.nx}x{g.ny} bc {g.bc_west}/{g.bc_east}: dL/d{name} rel L2 {err:.2e}")
            assert err < REL_GRAD
            assert np.all(got[c][s] == 0.0)


@pytest.mark.parametrize("nsteps,every", [(8, 8), (10, 3), (32, 8)])
def test_rollout_gradient_matches_fp64_reference(nsteps, every):
    _requires_gpu()
    _check(_gpu_and_reference(_batch(), nsteps, every, neq_mode=1), f"n={nsteps} K={every}")


@pytest.mark.parametrize("neq_mode", [0, 1])
def test_reinit_and_moments_adjoint_without_steps(neq_mode):
    """n = 0: the loss right after the reinit exercises the moment seed, the Zou-He
    transpose and the transposed difference stencils alone."""
    _requires_gpu()
    _check(_gpu_and_reference(_batch(), 0, 8, neq_mode), f"n=0 neq={neq_mode}")


def test_checkpoint_interval_does_not_change_the_gradient():
    _requires_gpu()
    specs = _batch()[:2]
    a = _gpu_and_reference(specs, 12, 1, 1)
    b = _gpu_and_reference(specs, 12, 12, 1)
    for (_, _, ga, _), (_, _, gb, _) in zip(a, b):
        for c in range(3):
            np.testing.assert_array_equal(ga[c], gb[c])
