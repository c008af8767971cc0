"""GPU parity of the hybrid FNO-LBM driver (Sec. 2.3, Fig. 3) against the oracle drivers."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300.fno import Fno, FnoShape, Hybrid, HybridConfig  # noqa: E402
from paper_2604_27158_gb300.lbm import GridSpec, Lattice  # noqa: E402

_, _, W, _ = oracle.lattice()


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def to_oracle(g):
    return oracle.Grid(nx=g.nx, ny=g.ny, tau=g.tau, fx=g.fx, fy=g.fy, bc_west=g.bc_west,
                       bc_east=g.bc_east, west_value=g.west_value, east_value=g.east_value)


def _net(width=8, layers=1, modes=3, seed=0, out_scale=1e-2):
    s = synth.FnoShape(width=width, layers=layers, modes=modes, dec_size=width)
    g = FnoShape(width=width, layers=layers, modes=modes, dec_size=width)
    params = synth.fno_random_params(s, seed=seed, out_scale=out_scale)
    return s, params, Fno(g, synth.fno_flatten_params(s, params))


def _porous(n, nx=64, ny=32):
    specs = []
    for k in range(n):
        solid, _, _ = synth.porous_media(nx, ny, 3, 4, seed=10 + k)
        specs.append((GridSpec(nx, ny, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                               west_value=1.001, east_value=1.0), solid))
    return specs


@pytest.mark.parametrize("use_fno", [0, 1])
def test_steady_driver_matches_oracle(use_fno):
    _requires_gpu()
    specs = _porous(3)
    s, params, net = _net(out_scale=1.0)
    lat = Lattice([a for a, _ in specs], [b for _, b in specs])
    hyb = Hybrid(lat, net, HybridConfig(use_fno=use_fno, neq_mode=1, check_every=100, tol=1e-30,
                                        max_steps=300))
    st, first, res = hyb.advance()
    assert st.steps == 300 and st.converged == 0 and np.all(first == -1)
    parts = lat.split(lat.export_f().cpu(), per_cell=9)
    for k, (g, solid) in enumerate(specs):
        f, hist = oracle.hybrid_steady(to_oracle(g), solid, s, params, nsteps=300,
                                       check_every=100, use_fno=bool(use_fno))
        fl = ~solid
        e = rel_l2(parts[k].numpy()[:, fl], (f - W[:, None, None])[:, fl])
        print(f"steady use_fno={use_fno} grid {k}: rel L2 g {e:.3e}, residual gpu {res[k]:.4e} "
              f"oracle {hist[-1][1]:.4e}")
        assert e < (1e-5 if not use_fno else 2e-2)
        assert abs(res[k] - hist[-1][1]) / hist[-1][1] < (1e-3 if not use_fno else 5e-2)


def test_steady_driver_first_check_from_rest():
    """From rest the stored velocity is 0, so the first check's residual is exactly 1;
    the driver's fused check (statistics taken inside a step) keeps level 100."""
    _requires_gpu()
    specs = _porous(2, nx=48, ny=24)
    lat = Lattice([a for a, _ in specs], [b for _, b in specs])
    hyb = Hybrid(lat, None, HybridConfig(use_fno=0, check_every=100, tol=1e-30, max_steps=100))
    st, first, res = hyb.advance()
    assert st.steps == 100 and lat.steps_done() == 100
    np.testing.assert_array_equal(res, 1.0)
    ref = Lattice([a for a, _ in specs], [b for _, b in specs])
    ref.step(100)
    assert torch.equal(lat.get_state().cpu(), ref.get_state().cpu())


def test_steady_driver_reports_convergence():
    _requires_gpu()
    specs = _porous(2, nx=48, ny=24)
    lat = Lattice([a for a, _ in specs], [b for _, b in specs])
    hyb = Hybrid(lat, None, HybridConfig(use_fno=0, check_every=100, tol=1e-3, max_steps=20000))
    st, first, res = hyb.advance()
    assert st.converged == 1 and np.all(first > 0) and np.all(res < 1e-3)
    assert st.steps == first.max() and st.steps % 100 == 0


@pytest.mark.parametrize("k_lbm", [10, 7])
def test_unsteady_cycles_match_oracle(k_lbm):
    """Super-time-stepping over a batch of two grid sizes (one FNO call per size)."""
    _requires_gpu()
    specs = []
    for k, (nx, ny) in enumerate([(48, 24), (64, 32), (48, 24)]):
        solid, _ = synth.flow_past_disks(nx, ny, seed=k, rmax=4)
        specs.append((GridSpec(nx, ny, 0.6 + 0.05 * k, bc_west=P.BC_VELOCITY, bc_east=P.BC_PRESSURE,
                               west_value=0.03, east_value=1.0), solid))
    s, params, net = _net(out_scale=1e-1)
    lat = Lattice([a for a, _ in specs], [b for _, b in specs])
    hyb = Hybrid(lat, net, HybridConfig(mode=P._abi.HYBRID_UNSTEADY, k_lbm=k_lbm, m_fno=2,
                                        neq_mode=1))
    st, _, _ = hyb.advance(cycles=3)
    torch.cuda.synchronize()
    assert st.steps == 3 * k_lbm and st.fno_calls == 3 * 2 * 2
    rho, ux, uy = (lat.split(t.cpu()) for t in lat.macro())
    for k, (g, solid) in enumerate(specs):
        f0 = oracle.rest_state(to_oracle(g), solid)
        f = oracle.hybrid_unsteady(to_oracle(g), solid, s, params, f0, k_lbm=k_lbm, m_fno=2,
                                   cycles=3)
        orho, oux, ouy = oracle.macro(to_oracle(g), solid, f)
        fl = ~solid
        e = rel_l2(np.stack([ux[k].numpy()[fl], uy[k].numpy()[fl]]), np.stack([oux[fl], ouy[fl]]))
        print(f"unsteady k={k_lbm} grid {k}: rel L2 u {e:.3e}")
        assert e < 2e-2


def test_uneven_batch_super_time_stepping_matches_oracle():
    """The batched unsteady workload (four grid sizes, k = 50 LBM steps, m = 5 FNO steps,
    reinit) on one trajectory per size, against the oracle driver with the same weights."""
    _requires_gpu()
    batch = synth.unsteady_batch(24, seed=3)
    picked, seen = [], set()
    for t in batch:
        if (t["nx"], t["ny"]) not in seen:
            seen.add((t["nx"], t["ny"]))
            picked.append(t)
    assert len(picked) == 4
    grids = [GridSpec(t["nx"], t["ny"], t["tau"], bc_west=P.BC_VELOCITY, bc_east=P.BC_PRESSURE,
                      west_value=t["u_in"], east_value=1.0) for t in picked]
    s, params, net = _net(width=16, layers=1, modes=4, out_scale=1e-1)
    assert all(net.uses_tensor_cores(t["ny"], t["nx"]) for t in picked)
    lat = Lattice(grids, [t["solid"] for t in picked])
    hyb = Hybrid(lat, net, HybridConfig(mode=P._abi.HYBRID_UNSTEADY, k_lbm=50, m_fno=5, neq_mode=1))
    st, _, _ = hyb.advance(cycles=2)
    torch.cuda.synchronize()
    assert st.steps == 100 and st.fno_calls == 2 * 5 * 4
    _, ux, uy = (lat.split(t.cpu()) for t in lat.macro())
    for k, (g, t) in enumerate(zip(grids, picked)):
        og, solid = to_oracle(g), t["solid"]
        f = oracle.hybrid_unsteady(og, solid, s, params, oracle.rest_state(og, solid), k_lbm=50,
                                   m_fno=5, cycles=2)
        _, oux, ouy = oracle.macro(og, solid, f)
        fl = ~solid
        e = rel_l2(np.stack([ux[k].numpy()[fl], uy[k].numpy()[fl]]), np.stack([oux[fl], ouy[fl]]))
        print(f"uneven batch {g.nx}x{g.ny}: rel L2 u {e:.3e}")
        assert e < 2e-2


def _pair_nets(cin_r, cin_u, width=8, modes=3, padding=0, seed=0, out_scale=1e-1):
    sr = synth.FnoShape(c_in=cin_r, c_out=1, width=width, layers=1, modes=modes, dec_size=width,
                        padding=padding)
    su = synth.FnoShape(c_in=cin_u, c_out=2, width=width, layers=2, modes=modes, dec_size=width,
                        padding=padding)
    pr = synth.fno_random_params(sr, seed=seed, out_scale=out_scale)
    pu = synth.fno_random_params(su, seed=seed + 1, out_scale=out_scale)
    gr = Fno(FnoShape(c_in=cin_r, c_out=1, width=width, layers=1, modes=modes, dec_size=width,
                      padding=padding), synth.fno_flatten_params(sr, pr))
    gu = Fno(FnoShape(c_in=cin_u, c_out=2, width=width, layers=2, modes=modes, dec_size=width,
                      padding=padding), synth.fno_flatten_params(su, pu))
    return (sr, pr), (su, pu), gr, gu


def test_density_and_velocity_networks_steady_from_the_mask():
    """Porous-media model group: a density and a velocity network, each reading the mask
    only (in channels: 1), padding 9, steady driver."""
    _requires_gpu()
    specs = _porous(2)
    (sr, pr), (su, pu), gr, gu = _pair_nets(1, 1, padding=9, out_scale=1.0)
    lat = Lattice([a for a, _ in specs], [b for _, b in specs])
    hyb = Hybrid(lat, gr, HybridConfig(use_fno=1, neq_mode=1, check_every=100, tol=1e-30,
                                       max_steps=200, in_channels=8, in_channels_u=8), fno_u=gu)
    st, _, _ = hyb.advance()
    assert st.steps == 200 and st.fno_calls == 2
    parts = lat.split(lat.export_f().cpu(), per_cell=9)
    nets = ((sr, pr, (3,)), (su, pu, (3,)))
    for k, (g, solid) in enumerate(specs):
        f, _ = oracle.hybrid_steady(to_oracle(g), solid, None, None, nsteps=200, check_every=100,
                                    nets=nets)
        fl = ~solid
        e = rel_l2(parts[k].numpy()[:, fl], (f - W[:, None, None])[:, fl])
        print(f"two-network steady grid {k}: rel L2 g {e:.3e}")
        assert e < 2e-2


def test_density_and_velocity_networks_unsteady_periodic():
    """Shear-layer model group: density network on rho - 1, velocity network on (u_x, u_y),
    padding 9, on fully periodic grids of two sizes, k = 20 LBM steps + 1 FNO step."""
    _requires_gpu()
    specs = []
    for k, n in enumerate((32, 48)):
        specs.append((GridSpec(n, n, 0.6), np.zeros((n, n), dtype=bool)))
    (sr, pr), (su, pu), gr, gu = _pair_nets(1, 2, padding=9, seed=4)
    lat = Lattice([a for a, _ in specs], [b for _, b in specs])
    rho0, ux0, uy0 = [], [], []
    for k, (g, _) in enumerate(specs):
        r, u, v = synth.smooth_macro_fields(g.nx, g.ny, seed=60 + k, drho=1e-2, umax=0.05)
        rho0.append(r.ravel()); ux0.append(u.ravel()); uy0.append(v.ravel())
    fields = [torch.from_numpy(np.concatenate(a)).cuda() for a in (rho0, ux0, uy0)]
    lat.reinit(*fields, neq_mode=1)
    hyb = Hybrid(lat, gr, HybridConfig(mode=P._abi.HYBRID_UNSTEADY, k_lbm=20, m_fno=1, neq_mode=1,
                                       in_channels=1, in_channels_u=6), fno_u=gu)
    st, _, _ = hyb.advance(cycles=2)
    torch.cuda.synchronize()
    assert st.steps == 40 and st.fno_calls == 2 * 2 * 2
    _, ux, uy = (lat.split(t.cpu()) for t in lat.macro())
    nets = ((sr, pr, (0,)), (su, pu, (1, 2)))
    off = lat.cell_offsets
    for k, (g, solid) in enumerate(specs):
        og = to_oracle(g)
        f0 = oracle.reinit(og, solid, rho0[k].reshape(g.ny, g.nx).astype(np.float64),
                           ux0[k].reshape(g.ny, g.nx).astype(np.float64),
                           uy0[k].reshape(g.ny, g.nx).astype(np.float64), 1)
        f = oracle.hybrid_unsteady(og, solid, None, None, f0, k_lbm=20, m_fno=1, cycles=2,
                                   nets=nets)
        _, oux, ouy = oracle.macro(og, solid, f)
        e = rel_l2(np.stack([ux[k].numpy(), uy[k].numpy()]), np.stack([oux, ouy]))
        print(f"two-network unsteady {g.nx}x{g.ny}: rel L2 u {e:.3e}")
        assert e < 2e-2


def test_unsteady_cycles_with_persistent_lbm_steps_are_identical():
    """The cycle's k LBM steps as one persistent launch (captured into the cycle's CUDA
    graph) give bitwise the same state as one launch per step."""
    _requires_gpu()
    specs = []
    for k, (nx, ny) in enumerate([(48, 24), (64, 32), (48, 24)]):
        solid, _ = synth.flow_past_disks(nx, ny, seed=k, rmax=4)
        specs.append((GridSpec(nx, ny, 0.6 + 0.05 * k, bc_west=P.BC_VELOCITY, bc_east=P.BC_PRESSURE,
                               west_value=0.03, east_value=1.0), solid))
    s, params, net = _net(out_scale=1e-1)
    states = []
    for persistent in (False, True):
        lat = Lattice([a for a, _ in specs], [b for _, b in specs])
        lat.set_persistent(persistent)
        hyb = Hybrid(lat, net, HybridConfig(mode=P._abi.HYBRID_UNSTEADY, k_lbm=7, m_fno=2,
                                            neq_mode=1))
        hyb.advance(cycles=3)
        torch.cuda.synchronize()
        states.append(lat.get_state().cpu())
    assert torch.equal(states[0], states[1])
