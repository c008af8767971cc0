"""GPU parity of the LBM kernels against the FP64 oracle, through the C ABI.

Bars: streaming / bounce-back index maps and masks bit-exact; FP32 fields
within 1e-5 relative L2 of the FP64 oracle after 1000 steps.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300.lbm import GridSpec, Lattice  # noqa: E402

_, _, W, _ = oracle.lattice()
REL_L2_FIELDS = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_oracle(g: GridSpec) -> oracle.Grid:
    return oracle.Grid(nx=g.nx, ny=g.ny, tau=g.tau, fx=g.fx, fy=g.fy, bc_west=g.bc_west,
                       bc_east=g.bc_east, west_value=g.west_value, east_value=g.east_value)


def probe_state(ny, nx, base=0):
    cell = np.arange(ny * nx).reshape(ny, nx)
    return (9 * (cell[None] + base) + np.arange(9)[:, None, None]).astype(np.float64)


def zou_he_unknown(g: GridSpec, solid):
    """bool [9, ny, nx]: populations completed by Zou-He (not a pure streaming value)."""
    m = np.zeros((9, g.ny, g.nx), bool)
    if g.bc_west != P.BC_PERIODIC:
        for i in (1, 5, 8):
            m[i, :, 0] = ~solid[:, 0]
        for i in (3, 6, 7):
            m[i, :, -1] = ~solid[:, -1]
    return m


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


GEOMS = {
    "channel_disks_40x24": lambda: (GridSpec(40, 24, 0.8), synth.channel_with_disks(40, 24, 3, 3, 5, seed=4)[0]),
    "ragged_37x21_periodic": lambda: (GridSpec(37, 21, 0.7),
                                      synth.rasterise_disks(37, 21, [synth.Disk(10, 7, 4), synth.Disk(30, 15, 3)], True, True)),
    "porous_zou_he_70x33": lambda: (GridSpec(70, 33, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                                             west_value=1.001, east_value=1.0),
                                    synth.porous_media(70, 33, 3, 5, seed=2)[0]),
    "velocity_inlet_64x32": lambda: (GridSpec(64, 32, 0.9, bc_west=P.BC_VELOCITY, bc_east=P.BC_PRESSURE,
                                              west_value=0.03, east_value=1.0),
                                     synth.flow_past_disks(64, 32, seed=1, rmax=6)[0]),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_streaming_index_map_bit_exact(name):
    _requires_gpu()
    g, solid = GEOMS[name]()
    lat = Lattice([g], [solid])
    fs = probe_state(g.ny, g.nx)
    lat.set_state(torch.from_numpy(fs.astype(np.float32).ravel()).cuda())
    got = lat.export_f().cpu().numpy().reshape(9, g.ny, g.nx).astype(np.float64)
    want = oracle.stream(to_oracle(g), solid, fs)
    known = ~zou_he_unknown(g, solid)
    fl = np.broadcast_to(~solid, want.shape)
    sel = known & fl
    np.testing.assert_array_equal(got[sel], want[sel])
    assert np.all(got[:, solid] == 0.0)  # solid cells export 0 (mask read exactly)
    # the state round-trips exactly
    np.testing.assert_array_equal(lat.get_state().cpu().numpy(), fs.astype(np.float32).ravel())


def test_streaming_index_map_batch_of_uneven_grids():
    _requires_gpu()
    specs = [GEOMS[k]() for k in sorted(GEOMS)]
    lat = Lattice([s[0] for s in specs], [s[1] for s in specs])
    parts, base = [], 0
    for g, _ in specs:
        parts.append(probe_state(g.ny, g.nx, base).ravel())
        base += g.nx * g.ny
    lat.set_state(torch.from_numpy(np.concatenate(parts).astype(np.float32)).cuda())
    got = lat.split(lat.export_f().cpu(), per_cell=9)
    base = 0
    for k, (g, solid) in enumerate(specs):
        want = oracle.stream(to_oracle(g), solid, probe_state(g.ny, g.nx, base))
        sel = ~zou_he_unknown(g, solid) & np.broadcast_to(~solid, want.shape)
        np.testing.assert_array_equal(got[k].numpy().astype(np.float64)[sel], want[sel])
        base += g.nx * g.ny


def _run_both(g, solid, steps, init="rest", seed=0):
    og = to_oracle(g)
    lat = Lattice([g], [solid])
    if init == "rest":
        f = oracle.rest_state(og, solid)
    else:
        rho, ux, uy = synth.smooth_macro_fields(g.nx, g.ny, seed=seed, drho=1e-3, umax=0.02)
        rho = rho.astype(np.float32)
        ux = ux.astype(np.float32)
        uy = uy.astype(np.float32)
        f = oracle.reinit(og, solid, rho, ux, uy, neq_mode=1)
        lat.reinit(*(torch.from_numpy(a.ravel()).cuda() for a in (rho, ux, uy)), neq_mode=1)
    f = oracle.run(og, solid, f, steps)
    lat.step(steps)
    torch.cuda.synchronize()
    gg = lat.export_f().cpu().numpy().reshape(9, g.ny, g.nx)
    rho, ux, uy = (t.cpu().numpy().reshape(g.ny, g.nx) for t in lat.macro())
    orho, oux, ouy = oracle.macro(og, solid, f)
    return lat, f, gg, (rho, ux, uy), (orho, oux, ouy)


def test_config1_channel_1000_and_2000_steps():
    """128x64 periodic channel, tau=0.8, gx=1e-6, 6 disks r 4-8, rest start."""
    _requires_gpu()
    solid, _ = synth.channel_with_disks(128, 64, 6, 4, 8, seed=0)
    g = GridSpec(128, 64, 0.8, fx=1e-6)
    for steps in (1000, 2000):
        lat, f, gg, (rho, ux, uy), (orho, oux, ouy) = _run_both(g, solid, steps)
        fl = ~solid
        e_u = rel_l2(np.stack([ux[fl], uy[fl]]), np.stack([oux[fl], ouy[fl]]))
        e_g = rel_l2(gg[:, fl], (f - W[:, None, None])[:, fl])
        e_rho = rel_l2(rho[fl], orho[fl])
        print(f"config1 steps={steps}: rel L2 u={e_u:.3e} g={e_g:.3e} rho={e_rho:.3e}")
        assert e_u < REL_L2_FIELDS and e_g < REL_L2_FIELDS and e_rho < REL_L2_FIELDS
        # invariants: mass exactly conserved by the oracle, to FP32 round-off by the GPU
        stats = lat.residual()
        assert abs(stats[0, P._abi.LBM_STAT_MASS] - orho[fl].sum()) / orho[fl].sum() < 1e-7
        mx = (orho * oux)[fl].sum()
        assert abs(stats[0, P._abi.LBM_STAT_MOMX] - mx) / abs(mx) < 1e-4


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_fields_1000_steps_from_reinit(name):
    """Decaying initial-value flows: the velocity decays ~100x over 1000 steps while
    FP32 storage rounding is committed in proportion to the field at each step, so
    the error is normalised by the initial field magnitude (the 1e-5 bar), and
    must also stay within 1e-4 of the final field."""
    _requires_gpu()
    g, solid = GEOMS[name]()
    _, f, gg, (rho, ux, uy), (orho, oux, ouy) = _run_both(g, solid, 1000, init="fields", seed=3)
    _, ux0, uy0 = synth.smooth_macro_fields(g.nx, g.ny, seed=3, drho=1e-3, umax=0.02)
    fl = ~solid
    du = np.stack([ux[fl] - oux[fl], uy[fl] - ouy[fl]])
    e_u0 = float(np.linalg.norm(du) / np.linalg.norm(np.stack([ux0[fl], uy0[fl]])))
    e_u = rel_l2(np.stack([ux[fl], uy[fl]]), np.stack([oux[fl], ouy[fl]]))
    e_g = rel_l2(gg[:, fl], (f - W[:, None, None])[:, fl])
    print(f"{name}: error/|u0|={e_u0:.3e} rel L2 u={e_u:.3e} g={e_g:.3e}")
    assert e_u0 < REL_L2_FIELDS and e_u < 10 * REL_L2_FIELDS and e_g < 10 * REL_L2_FIELDS


def test_config2_porous_512x256_1000_steps():
    """Full-size porous medium (pressure inlet 1.001 / outlet 1.0, tau 0.7, r 4-12)."""
    _requires_gpu()
    solid, _, phi = synth.porous_media(512, 256, 4, 12, seed=0)
    assert 0.6 <= phi <= 0.8
    g = GridSpec(512, 256, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE, west_value=1.001,
                 east_value=1.0)
    lat, f, gg, (rho, ux, uy), (orho, oux, ouy) = _run_both(g, solid, 1000)
    fl = ~solid
    e_u = rel_l2(np.stack([ux[fl], uy[fl]]), np.stack([oux[fl], ouy[fl]]))
    e_drho = rel_l2(rho[fl] - 1.0, orho[fl] - 1.0)
    print(f"config2 1000 steps: rel L2 u={e_u:.3e} drho={e_drho:.3e}")
    assert e_u < REL_L2_FIELDS and e_drho < 1e-4
    st = lat.residual()
    dp_or = ((orho[:, 0][fl[:, 0]]).mean() - (orho[:, -1][fl[:, -1]]).mean()) / 3.0
    assert abs(st[0, P._abi.LBM_STAT_DP] - dp_or) / dp_or < 1e-5


def test_reinit_matches_oracle():
    _requires_gpu()
    g, solid = GEOMS["porous_zou_he_70x33"]()
    rho, ux, uy = (a.astype(np.float32) for a in synth.smooth_macro_fields(g.nx, g.ny, seed=9))
    for neq in (0, 1):
        lat = Lattice([g], [solid])
        lat.reinit(*(torch.from_numpy(a.ravel()).cuda() for a in (rho, ux, uy)), neq_mode=neq)
        gg = lat.export_f().cpu().numpy().reshape(9, g.ny, g.nx)
        f = oracle.reinit(to_oracle(g), solid, rho, ux, uy, neq_mode=neq)
        fl = ~solid
        e = rel_l2(gg[:, fl], (f - W[:, None, None])[:, fl])
        assert e < 1e-6, (neq, e)
        # the stored slots of solid cells hold g = 0 (no pull reads them)
        raw = lat.get_state().cpu().numpy().reshape(9, g.ny, g.nx)
        assert np.all(raw[:, solid] == 0.0)


def test_residual_statistics_match_oracle():
    _requires_gpu()
    g, solid = GEOMS["porous_zou_he_70x33"]()
    og = to_oracle(g)
    lat = Lattice([g], [solid])
    lat.step(100)
    lat.residual(update_prev=True)
    f = oracle.run(og, solid, oracle.rest_state(og, solid), 100)
    _, ux0, uy0 = oracle.macro(og, solid, f)
    lat.step(100)
    st = lat.residual(update_prev=True)[0]
    f = oracle.run(og, solid, f, 100)
    rho1, ux1, uy1 = oracle.macro(og, solid, f)
    r = oracle.steady_residual(solid, ux1, uy1, ux0, uy0)
    assert abs(st[P._abi.LBM_STAT_RESIDUAL] - r) / r < 1e-4
    assert st[P._abi.LBM_STAT_FLUID] == (~solid).sum()
    assert st[P._abi.LBM_STAT_BAD] == 0


def test_unstable_state_is_reported():
    _requires_gpu()
    g = GridSpec(32, 16, 0.8)
    solid = np.zeros((16, 32), bool)
    lat = Lattice([g], [solid], u_max=0.1)
    rho = torch.ones(32 * 16, device="cuda")
    ux = torch.full_like(rho, 0.15)   # above u_max
    uy = torch.zeros_like(rho)
    lat.reinit(rho, ux, uy, neq_mode=0)
    with pytest.raises(P.LbmError) as e:
        lat.residual()
    assert e.value.code == P._abi.LBM_ERR_UNSTABLE
    st = lat.residual(raise_unstable=False)
    assert st[0, P._abi.LBM_STAT_BAD] == 32 * 16


def test_degenerate_grids():
    _requires_gpu()
    # smallest lattice, an all-solid lattice and a lattice one cell past a word boundary
    specs = [(GridSpec(2, 2, 0.8), np.zeros((2, 2), bool)),
             (GridSpec(8, 4, 0.8), np.ones((4, 8), bool)),
             (GridSpec(33, 3, 0.6), np.zeros((3, 33), bool))]
    lat = Lattice([s[0] for s in specs], [s[1] for s in specs])
    lat.step(10)
    st = lat.residual(update_prev=False)
    assert st[1, P._abi.LBM_STAT_FLUID] == 0
    gg = lat.split(lat.export_f().cpu(), per_cell=9)
    assert torch.all(gg[0] == 0) and torch.all(gg[1] == 0) and torch.all(gg[2] == 0)


def test_all_step_tile_shapes_give_identical_states():
    """Every compiled tile shape runs the same per-cell arithmetic: states agree bitwise."""
    _requires_gpu()
    specs = [GEOMS[k]() for k in sorted(GEOMS)]
    solid2, _, _ = synth.porous_media(512, 256, 4, 12, seed=5)
    specs.append((GridSpec(512, 256, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                           west_value=1.001, east_value=1.0), solid2))
    ref = None
    for v in range(P._abi.LBM_STEP_VARIANTS):
        lat = Lattice([s[0] for s in specs], [s[1] for s in specs])
        try:
            lat.set_step_variant(v)
        except P.LbmError:
            continue  # a shape that does not fit on this device
        lat.step(37)
        state = lat.get_state().cpu()
        if ref is None:
            ref = state
        else:
            assert torch.equal(state, ref), f"tile shape {v} differs"
    assert ref is not None


def test_autotune_keeps_state_and_picks_a_shape():
    _requires_gpu()
    g, solid = GEOMS["porous_zou_he_70x33"]()
    lat = Lattice([g], [solid])
    lat.step(11)
    before = lat.get_state().cpu()
    chosen, ms = lat.autotune(reps=3)
    assert torch.equal(lat.get_state().cpu(), before)
    assert 0 <= chosen < P._abi.LBM_STEP_VARIANTS and ms[chosen] == min(ms)
    assert lat.step_variant()[0] == chosen
    lat.step(5)
    ref = Lattice([g], [solid])
    ref.step(16)
    assert torch.equal(lat.get_state().cpu(), ref.get_state().cpu())


# ---------------------------------------------------------------------------
# The index map of the kernel that advances the lattice.  lbm_stream_probe runs the
# step kernel (the same cp.async.bulk row staging, +-1 shifts across 16-byte chunks,
# funnel-shifted mask windows, wrap columns and short last tiles) with the collision
# replaced by the identity, so the stored state becomes the streamed populations.
# With the index-valued probe state every value is an exact integer in FP32: the
# moved values must equal the oracle's streaming (Sec. 2.1) bit for bit.

def _probe_specs():
    specs = [GEOMS[k]() for k in sorted(GEOMS)]
    solid, _, _ = synth.porous_media(512, 256, 4, 12, seed=7)       # 4 x-tiles, Zou-He ends
    specs.append((GridSpec(512, 256, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                           west_value=1.001, east_value=1.0), solid))
    # periodic, 3 x-tiles with a ragged last one (301 = 2 * 128 + 45), ny prime
    solid = synth.rasterise_disks(301, 23, [synth.Disk(0, 5, 4), synth.Disk(300, 17, 3),
                                            synth.Disk(128, 11, 5), synth.Disk(255, 0, 3)],
                                  True, True)
    specs.append((GridSpec(301, 23, 0.8), solid))
    return specs


def _check_streamed(specs, got_parts, base0=0):
    base = base0
    for k, (g, solid) in enumerate(specs):
        fs = probe_state(g.ny, g.nx, base)
        want = oracle.stream(to_oracle(g), solid, fs)
        got = got_parts[k].numpy().astype(np.float64).reshape(9, g.ny, g.nx)
        sel = ~zou_he_unknown(g, solid) & np.broadcast_to(~solid, want.shape)
        np.testing.assert_array_equal(got[sel], want[sel], err_msg=f"grid {k} {g.nx}x{g.ny}")
        assert np.all(got[:, solid] == 0.0), f"grid {k}: solid cells must store 0"
        base += g.nx * g.ny


@pytest.mark.parametrize("variant", range(6))
def test_step_kernel_streaming_bit_exact_every_tile_shape(variant):
    _requires_gpu()
    assert P._abi.LBM_STEP_VARIANTS == 6
    specs = _probe_specs()
    # each grid alone (one launch covers one geometry) ...
    for g, solid in specs:
        lat = Lattice([g], [solid])
        lat.set_state(torch.from_numpy(probe_state(g.ny, g.nx).astype(np.float32).ravel()).cuda())
        lat.stream_probe(variant)
        _check_streamed([(g, solid)], [lat.get_state().cpu()])
        lat.close()
    # ... and all of them as one batch of uneven grids
    lat = Lattice([s[0] for s in specs], [s[1] for s in specs])
    parts, base = [], 0
    for g, _ in specs:
        parts.append(probe_state(g.ny, g.nx, base).ravel())
        base += g.nx * g.ny
    assert 9 * base < 2 ** 24  # every probe value is exact in FP32
    lat.set_state(torch.from_numpy(np.concatenate(parts).astype(np.float32)).cuda())
    lat.stream_probe(variant)
    _check_streamed(specs, lat.split(lat.get_state().cpu(), per_cell=9))
    lat.close()


def test_stream_probe_equals_export_on_moved_values():
    """The step kernel's gather and the per-cell gather of lbm_export_f agree."""
    _requires_gpu()
    specs = _probe_specs()
    lat = Lattice([s[0] for s in specs], [s[1] for s in specs])
    rng = np.random.default_rng(3)
    state = torch.from_numpy(rng.standard_normal(9 * lat.cells).astype(np.float32)).cuda()
    lat.set_state(state)
    exported = lat.export_f().cpu()
    lat.stream_probe(3)
    streamed = lat.get_state().cpu()
    for k, (g, solid) in enumerate(specs):
        a = lat.split(exported, per_cell=9)[k].numpy().reshape(9, g.ny, g.nx)
        b = lat.split(streamed, per_cell=9)[k].numpy().reshape(9, g.ny, g.nx)
        known = ~zou_he_unknown(g, solid)
        np.testing.assert_array_equal(a[known], b[known])
        # the Zou-He unknowns: the same FP32 formula, up to rounding order
        np.testing.assert_allclose(a[~known], b[~known], rtol=1e-5, atol=1e-6)


# ---------------------------------------------------------------------------
# Statistics taken by the step kernel (stats-only mode for lbm_residual, step + stats
# for lbm_step_residual and the steady driver).

def _stats_lattice():
    specs = _probe_specs()
    specs.append((GridSpec(128, 64, 0.8, fx=1e-6), synth.channel_with_disks(128, 64, 6, 4, 8, seed=0)[0]))
    return specs


def test_residual_identical_for_every_tile_shape():
    _requires_gpu()
    specs = _stats_lattice()
    ref = None
    for v in range(P._abi.LBM_STEP_VARIANTS):
        lat = Lattice([s[0] for s in specs], [s[1] for s in specs])
        lat.set_step_variant(v)
        lat.step(60)
        lat.residual(update_prev=True)
        lat.step(40)
        st = lat.residual(update_prev=False)
        if ref is None:
            ref = st
        else:  # same per-segment FP32 trees and the same FP64 order in every shape
            np.testing.assert_array_equal(st, ref, err_msg=f"tile shape {v}")
        lat.close()
    assert np.all(ref[:, P._abi.LBM_STAT_RESIDUAL] > 0)


@pytest.mark.parametrize("variant", [0, 3])
def test_step_residual_equals_residual_then_step(variant):
    _requires_gpu()
    specs = _stats_lattice()
    a = Lattice([s[0] for s in specs], [s[1] for s in specs])
    b = Lattice([s[0] for s in specs], [s[1] for s in specs])
    for lat in (a, b):
        lat.set_step_variant(variant)
        lat.step(50)
        lat.residual(update_prev=True)
        lat.step(25)
    for _ in range(3):
        sa = a.step_residual(update_prev=True)
        sb = b.residual(update_prev=True)
        b.step(1)
        np.testing.assert_array_equal(sa, sb)
        assert torch.equal(a.get_state().cpu(), b.get_state().cpu())
        a.step(9)
        b.step(9)
    assert a.steps_done() == b.steps_done()
    np.testing.assert_array_equal(a.residual(update_prev=False), b.residual(update_prev=False))


# ---------------------------------------------------------------------------
# Persistent multi-step launch: nsteps in one cooperative launch with a grid-wide
# barrier between steps.

@pytest.mark.parametrize("variant", range(6))
def test_persistent_steps_bitwise_equal_one_launch_per_step(variant):
    _requires_gpu()
    specs = _stats_lattice()
    a = Lattice([s[0] for s in specs], [s[1] for s in specs])
    b = Lattice([s[0] for s in specs], [s[1] for s in specs])
    for lat in (a, b):
        lat.set_step_variant(variant)
    a.set_persistent(True)
    for n in (37, 100, 1, 2):   # odd and even counts; a single step takes one launch
        a.step(n)
        b.step(n)
        assert torch.equal(a.get_state().cpu(), b.get_state().cpu()), f"after {n} steps"
    assert a.steps_done() == b.steps_done() == 140
    np.testing.assert_array_equal(a.residual(update_prev=False), b.residual(update_prev=False))


def test_persistent_barrier_selftest_expires_and_context_stays_usable():
    """The grid barrier's bounded wait: a barrier that waits for one CTA more than the
    launch has expires after the limit with LBM_ERR_TIMEOUT and leaves the state as it
    was; the same launch with every CTA arriving completes; normal work follows."""
    _requires_gpu()
    g, solid = GEOMS["porous_zou_he_70x33"]()
    lat = Lattice([g], [solid])
    lat.step(10)
    before = lat.get_state().cpu()
    assert lat.barrier_selftest(arrive_all=False, limit_ms=5.0) == P._abi.LBM_ERR_TIMEOUT
    assert "grid barrier" in P._abi.last_error()
    assert torch.equal(lat.get_state().cpu(), before)
    assert lat.barrier_selftest(arrive_all=True, limit_ms=500.0) == P._abi.LBM_OK
    ref = Lattice([g], [solid])
    ref.step(12)
    assert torch.equal(lat.get_state().cpu(), ref.get_state().cpu())
    lat.set_persistent(True)
    lat.step(20)
    ref.step(20)
    assert torch.equal(lat.get_state().cpu(), ref.get_state().cpu())
    st = lat.residual()   # the step kernel's own status word is clean
    assert st[0, P._abi.LBM_STAT_BAD] == 0
