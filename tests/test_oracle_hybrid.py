"""Pins of the oracle's hybrid parts (Sec. 2.3, Fig. 3): the clamp of FNO predictions
before re-initialisation, and the order of the super-time-stepping cycle
(k LBM steps -> macroscopic fields -> m FNO steps -> re-initialisation).

The clamp is checked against hand-computed vectors and its geometric invariants
(direction kept, speed capped, density clipped on both sides), not against a retyped
formula.  The cycle is checked through special cases whose outcome is fixed without
running the driver's own sequence: a network with a constant output must leave the
re-initialised equilibrium of the clamped constant; with no FNO step a cycle is k LBM
steps and a re-initialisation that reproduces a smooth flow, so the cycles follow
plain LBM step for step; the steady driver's first residual from rest is exactly 1.
"""
import numpy as np
import pytest

import oracle
import synth

CX, CY, W, OPP = oracle.lattice()


# --------------------------------------------------------------------- clamp ---

def test_clamp_macro_known_vectors():
    rho = np.array([0.5, 0.95, 1.5, 1.1, 0.9])
    ux = np.array([0.3, 0.1, 0.0, -0.12, 0.0])
    uy = np.array([0.4, 0.1, -0.25, 0.16, 0.0])
    r, vx, vy = oracle.clamp_macro(rho, ux, uy, 0.9, 1.1, 0.2)
    # density clipped on both sides, untouched inside [0.9, 1.1]
    np.testing.assert_array_equal(r, [0.9, 0.95, 1.1, 1.1, 0.9])
    # |(0.3, 0.4)| = 0.5 -> scaled by 0.4 to (0.12, 0.16): the direction is kept, so a
    # component-wise clamp (which would give (0.2, 0.2)) fails here
    np.testing.assert_allclose([vx[0], vy[0]], [0.12, 0.16], rtol=1e-15)
    # below the cap: unchanged
    assert vx[1] == 0.1 and vy[1] == 0.1
    # one component above the cap
    np.testing.assert_allclose([vx[2], vy[2]], [0.0, -0.2], rtol=1e-15)
    # exactly at the cap (|(-0.12, 0.16)| = 0.2) and at rest: unchanged
    np.testing.assert_allclose([vx[3], vy[3]], [-0.12, 0.16], rtol=1e-15)
    assert vx[4] == 0.0 and vy[4] == 0.0


def test_clamp_macro_keeps_direction_and_caps_speed():
    rng = np.random.default_rng(0)
    ux, uy = rng.normal(0, 0.3, 1000), rng.normal(0, 0.3, 1000)
    rho = rng.uniform(0.5, 1.5, 1000)
    r, vx, vy = oracle.clamp_macro(rho, ux, uy, 0.9, 1.1, 0.2)
    sp, sp2 = np.hypot(ux, uy), np.hypot(vx, vy)
    np.testing.assert_allclose(sp2, np.minimum(sp, 0.2), rtol=1e-14)
    np.testing.assert_allclose(vx * uy - vy * ux, 0.0, atol=1e-15)   # parallel
    assert np.all(vx * ux + vy * uy >= 0)                            # same sense
    assert r.min() >= 0.9 and r.max() <= 1.1
    inside = (rho >= 0.9) & (rho <= 1.1)
    np.testing.assert_array_equal(r[inside], rho[inside])


# ------------------------------------------------------------- cycle order ---

def _periodic_with_disks(nx=40, ny=24, seed=3):
    solid = synth.rasterise_disks(nx, ny, [synth.Disk(12, 8, 4), synth.Disk(30, 17, 3)],
                                  True, True)
    return oracle.Grid(nx=nx, ny=ny, tau=0.8), solid


def test_unsteady_cycle_ends_with_reinit_of_the_clamped_fno_prediction():
    """A network whose output layer has zero weights predicts its bias everywhere.
    Whatever the LBM did before, every cycle must then end with the populations of the
    re-initialisation from the clamped constant: f^eq(rho_c, u_c) at every fluid cell
    (uniform fields have zero gradients, so f^neq vanishes)."""
    g, solid = _periodic_with_disks()
    shape = synth.FnoShape(width=8, layers=1, modes=3, dec_size=8)
    params = synth.fno_random_params(shape, seed=1)
    params["out.w"] = np.zeros_like(params["out.w"])
    params["out.b"] = np.array([0.25, 0.25, -0.5], np.float32)   # exact in bfloat16
    f0 = oracle.rest_state(g, solid)
    f = oracle.hybrid_unsteady(g, solid, shape, params, f0, k_lbm=7, m_fno=2, cycles=2)
    # clamp: rho = 1.25 -> 1.1; |u| = sqrt(0.3125) -> 0.2, same direction
    s = 0.2 / np.hypot(0.25, -0.5)
    feq = oracle.equilibrium(1.1, 0.25 * s, -0.5 * s)
    fl = ~solid
    np.testing.assert_allclose(f[:, fl], np.broadcast_to(feq[:, None], (9, fl.sum())),
                               rtol=0, atol=1e-15)
    # the statement is not empty: without the clamp or without the reinit it fails
    assert np.abs(oracle.equilibrium(1.25, 0.25, -0.5) - feq).max() > 1e-2


def _taylor_green(n=32, u0=0.02):
    x = np.arange(n)
    X, Y = np.meshgrid(x, x)
    k = 2 * np.pi / n
    ux = -u0 * np.cos(k * X) * np.sin(k * Y)
    uy = u0 * np.sin(k * X) * np.cos(k * Y)
    rho = 1.0 - 0.75 * u0 * u0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return rho, ux, uy


@pytest.mark.parametrize("k_lbm", [1, 4, 5])
def test_unsteady_cycles_without_fno_steps_follow_plain_lbm(k_lbm):
    """m = 0: a cycle is k LBM steps then a re-initialisation from the macroscopic
    fields with the Chapman-Enskog non-equilibrium estimate, which reproduces a smooth
    Taylor-Green flow to second order.  So `cycles` cycles follow plain LBM over
    k * cycles steps, much closer than the change made by one LBM step more or less:
    the number and place of the LBM steps in the cycle are pinned."""
    n = 32
    g = oracle.Grid(nx=n, ny=n, tau=0.8)
    solid = np.zeros((n, n), bool)
    rho, ux, uy = _taylor_green(n)
    f0 = oracle.reinit(g, solid, rho, ux, uy, neq_mode=1)
    cycles = 20 // k_lbm
    steps = k_lbm * cycles
    fh = oracle.hybrid_unsteady(g, solid, None, None, f0, k_lbm=k_lbm, m_fno=0, cycles=cycles)
    _, hx, hy = oracle.macro(g, solid, fh)

    def u_after(nsteps):
        _, vx, vy = oracle.macro(g, solid, oracle.run(g, solid, f0, nsteps))
        return np.stack([vx, vy])

    ref = u_after(steps)
    err = np.linalg.norm(np.stack([hx, hy]) - ref) / np.linalg.norm(ref)
    one_step = min(np.linalg.norm(u_after(steps + d) - ref) for d in (-1, 1)) / np.linalg.norm(ref)
    assert err < 0.25 * one_step, (err, one_step)


def test_steady_driver_first_residual_from_rest_is_one():
    """From rest the stored velocity is 0, so the first residual ||u - 0|| / ||u|| is 1
    exactly, at step check_every; later checks compare consecutive check levels."""
    solid, _, _ = synth.porous_media(nx=64, ny=32, rmin=3, rmax=4, seed=3)
    g = oracle.Grid(nx=64, ny=32, tau=0.7, bc_west=oracle.BC_PRESSURE,
                    bc_east=oracle.BC_PRESSURE, west_value=1.001, east_value=1.0)
    f, hist = oracle.hybrid_steady(g, solid, None, None, nsteps=250, check_every=100,
                                   use_fno=False)
    assert [h[0] for h in hist] == [100, 200, 250]
    assert hist[0][1] == 1.0
    rest = oracle.rest_state(g, solid)
    f200 = oracle.run(g, solid, rest, 200)
    f250 = oracle.run(g, solid, f200, 50)
    np.testing.assert_array_equal(f, f250)
    _, ax, ay = oracle.macro(g, solid, f200)
    _, bx, by = oracle.macro(g, solid, f250)
    fl = ~solid
    want = np.sqrt(((bx - ax)[fl] ** 2 + (by - ay)[fl] ** 2).sum() / (bx[fl] ** 2 + by[fl] ** 2).sum())
    assert abs(hist[2][1] - want) <= 1e-14 * want
