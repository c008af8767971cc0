"""GPU parts of the double-shear-layer workload (Sec. 3.2.1-3.2.2): the vorticity metric
against the oracle, the stability of the lattice set-up over the 30 Delta T horizon, and
a 1:1 hybrid cycle with the paper's density/velocity model pair (padding 9) against the
oracle driver."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300.fno import Fno, FnoShape, Hybrid, HybridConfig  # noqa: E402
from paper_2604_27158_gb300.lbm import GridSpec, Lattice  # noqa: E402


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def to_oracle(g):
    return oracle.Grid(nx=g.nx, ny=g.ny, tau=g.tau, fx=g.fx, fy=g.fy, bc_west=g.bc_west,
                       bc_east=g.bc_east, west_value=g.west_value, east_value=g.east_value)


def test_vorticity_matches_oracle():
    _requires_gpu()
    specs = []
    s, _, _ = synth.porous_media(64, 32, 3, 4, seed=1)
    specs.append((GridSpec(64, 32, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                           west_value=1.01, east_value=1.0), s))
    specs.append((GridSpec(40, 24, 0.6), np.zeros((24, 40), bool)))
    s, _ = synth.channel_with_disks(48, 24, 2, 2, 3, seed=2)
    specs.append((GridSpec(48, 24, 0.8, fx=1e-5), s))
    lat = Lattice([g for g, _ in specs], [m for _, m in specs])
    fields = [synth.smooth_macro_fields(g.nx, g.ny, seed=k, umax=0.05) for k, (g, _) in
              enumerate(specs)]
    ux = torch.from_numpy(np.concatenate([f[1].ravel() for f in fields])).cuda()
    uy = torch.from_numpy(np.concatenate([f[2].ravel() for f in fields])).cuda()
    w = lat.split(lat.vorticity(ux, uy).cpu())
    for k, (g, solid) in enumerate(specs):
        ref = oracle.vorticity(to_oracle(g), solid, fields[k][1], fields[k][2])
        e = rel_l2(w[k].numpy(), ref)
        print(f"vorticity {g.nx}x{g.ny}: rel L2 {e:.2e}")
        assert e < 1e-6
        assert np.all(w[k].numpy()[solid] == 0.0)


def test_double_shear_lattice_set_up_is_stable_over_the_horizon():
    """128^2 periodic, tau = 1/2 + 3 nu dt/dx^2, U in lattice units = U dt/dx: 30 Delta T
    (6690 steps) of pure LBM from the sharpest and the smoothest layers stay finite and
    conserve mass."""
    _requires_gpu()
    setup = synth.DoubleShear()
    ics = synth.double_shear(2, seed=5, a_range=(125.0, 125.0)) + \
        synth.double_shear(2, seed=6, a_range=(20.0, 20.0))
    n = setup.n
    lat = Lattice([GridSpec(n, n, setup.tau)] * 4, [np.zeros((n, n), bool)] * 4, u_max=0.3)
    fields = [torch.from_numpy(np.concatenate([ic[k].ravel() for ic in ics])).cuda()
              for k in ("rho", "ux", "uy")]
    lat.reinit(*fields, neq_mode=1)
    m0 = lat.residual(update_prev=True)[:, P._abi.LBM_STAT_MASS].copy()
    lat.step(30 * setup.steps_per_dT)
    st = lat.residual(update_prev=True)
    assert np.all(st[:, P._abi.LBM_STAT_BAD] == 0)
    np.testing.assert_allclose(st[:, P._abi.LBM_STAT_MASS], m0, rtol=1e-5)


def test_double_shear_hybrid_cycle_matches_oracle():
    """One 1:1 cycle (223 LBM steps, then one FNO step of a density network on rho - 1
    and a velocity network on (u_x, u_y), padding 9, then reinit) on two trajectories."""
    _requires_gpu()
    setup = synth.DoubleShear()
    n = setup.n
    ics = synth.double_shear(2, seed=9)
    sr = synth.FnoShape(c_in=1, c_out=1, width=8, layers=2, modes=8, dec_size=16, padding=9)
    su = synth.FnoShape(c_in=2, c_out=2, width=8, layers=2, modes=16, dec_size=16, padding=9)
    pr = synth.fno_random_params(sr, seed=1, out_scale=1e-2)
    pu = synth.fno_random_params(su, seed=2, out_scale=1e-2)
    gr = Fno(FnoShape(c_in=1, c_out=1, width=8, layers=2, modes=8, dec_size=16, padding=9),
             synth.fno_flatten_params(sr, pr))
    gu = Fno(FnoShape(c_in=2, c_out=2, width=8, layers=2, modes=16, dec_size=16, padding=9),
             synth.fno_flatten_params(su, pu))
    g = GridSpec(n, n, setup.tau)
    lat = Lattice([g, g], [np.zeros((n, n), bool)] * 2, u_max=0.3)
    fields = [torch.from_numpy(np.concatenate([ic[k].ravel() for ic in ics])).cuda()
              for k in ("rho", "ux", "uy")]
    lat.reinit(*fields, neq_mode=1)
    hyb = Hybrid(lat, gr, HybridConfig(mode=P._abi.HYBRID_UNSTEADY, k_lbm=setup.steps_per_dT,
                                       m_fno=1, neq_mode=1, in_channels=1, in_channels_u=6),
                 fno_u=gu)
    hyb.advance(cycles=1)
    torch.cuda.synchronize()
    _, ux, uy = (lat.split(t.cpu()) for t in lat.macro())
    nets = ((sr, pr, (0,)), (su, pu, (1, 2)))
    og = to_oracle(g)
    solid = np.zeros((n, n), bool)
    for k, ic in enumerate(ics):
        f0 = oracle.reinit(og, solid, ic["rho"].astype(np.float64), ic["ux"].astype(np.float64),
                           ic["uy"].astype(np.float64), 1)
        f = oracle.hybrid_unsteady(og, solid, None, None, f0, k_lbm=setup.steps_per_dT, m_fno=1,
                                   cycles=1, nets=nets)
        _, oux, ouy = oracle.macro(og, solid, f)
        e = rel_l2(np.stack([ux[k].numpy(), uy[k].numpy()]), np.stack([oux, ouy]))
        print(f"double shear 1:1 cycle, trajectory {k}: rel L2 u {e:.3e}")
        assert e < 2e-2
