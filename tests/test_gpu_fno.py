"""GPU parity of the FNO forward pass (Sec. 2.2) against the FP64 oracle, through the C ABI.

Bar: BF16 FNO outputs within 2e-2 relative L2 of the FP64 oracle, which sees the
same bfloat16-rounded parameters and inputs.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import fno_oracle as fo

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300.fno import Fno, FnoShape  # noqa: E402

REL_L2_FNO = 2e-2


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _pair(c_in=4, c_out=3, width=8, layers=2, modes=3, dec_layers=1, dec_size=8, act=0, seed=1,
          out_scale=1.0):
    s = synth.FnoShape(c_in=c_in, c_out=c_out, width=width, layers=layers, modes=modes,
                       dec_layers=dec_layers, dec_size=dec_size)
    g = FnoShape(c_in=c_in, c_out=c_out, width=width, layers=layers, modes=modes,
                 dec_layers=dec_layers, dec_size=dec_size, activation=act)
    params = synth.fno_random_params(s, seed=seed, out_scale=out_scale)
    return s, g, params


def _inputs(B, c_in, H, W, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, c_in, H, W)).astype(np.float32)


@pytest.mark.parametrize("B,H,W,act", [(2, 12, 16, 0), (1, 6, 7, 1), (3, 20, 33, 0)])
def test_small_fno_matches_oracle(B, H, W, act):
    _requires_gpu()
    s, g, params = _pair(act=act)
    net = Fno(g, synth.fno_flatten_params(s, params))
    x = _inputs(B, 4, H, W, seed=B + H)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = fo.fno_forward(s, params, x, activation="gelu" if act == 0 else "relu")
    e = rel_l2(y, ref)
    print(f"FNO {B}x{H}x{W} act={act}: rel L2 {e:.3e}")
    assert e < REL_L2_FNO


@pytest.mark.parametrize("width,modes,dec_layers,H,W", [
    (48, 5, 1, 24, 40),    # C > 32: the frequency-parallel x/y kernels, k_inv_x_row<64>
    (24, 16, 1, 40, 36),   # 2m >= 32: the row-parallel forward y-DFT, C <= 32 row kernels
    (16, 4, 2, 18, 22),    # two hidden decoder layers: the general projection kernel
])
def test_cuda_core_kernel_variants_match_oracle(width, modes, dec_layers, H, W):
    """Each CUDA-core kernel variant the dispatcher picks by channel count, mode count
    and decoder depth, against the FP64 oracle (path forced to CUDA cores)."""
    _requires_gpu()
    s, g, params = _pair(width=width, layers=2, modes=modes, dec_layers=dec_layers,
                         dec_size=20, seed=width + modes)
    net = Fno(g, synth.fno_flatten_params(s, params))
    net.set_path(P._abi.FNO_PATH_CUDA_CORES)
    x = _inputs(2, 4, H, W, seed=width)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    e = rel_l2(y, fo.fno_forward(s, params, x))
    print(f"FNO CUDA cores C={width} m={modes} dec={dec_layers} {H}x{W}: rel L2 {e:.3e}")
    assert e < REL_L2_FNO


@pytest.mark.parametrize("H,W", [(32, 48), (64, 64)])
def test_hot_path_architecture_matches_oracle(H, W):
    """4 layers, 32 latent channels, 12x12 modes, decoder 32 -> 3 (2,365,331 parameters)."""
    _requires_gpu()
    s, g, params = _pair(width=32, layers=4, modes=12, dec_size=32, seed=5)
    assert fo.param_count(s) == 2365331
    net = Fno(g, synth.fno_flatten_params(s, params))
    x = _inputs(2, 4, H, W, seed=7)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = fo.fno_forward(s, params, x)
    e = rel_l2(y, ref)
    print(f"FNO C=32 m=12 {H}x{W}: rel L2 {e:.3e}")
    assert e < REL_L2_FNO


def _flow_inputs(B, H, W, seed0=0):
    """(rho-1, ux, uy, mask) shaped like snapshots of the 128x64 channel workload, at H x W."""
    xs = []
    for b in range(B):
        solid, _ = synth.channel_with_disks(W, H, 6, 4 * W // 128, 8 * W // 128, seed=seed0 + b)
        rho, ux, uy = synth.smooth_macro_fields(W, H, seed=seed0 + b, drho=1e-3, umax=0.05)
        f = np.stack([rho - 1.0, ux, uy, solid.astype(np.float32)]).astype(np.float32)
        f[:3, solid] = 0.0
        xs.append(f)
    return np.stack(xs)


def test_fno_throughput_workload_sampled_against_oracle():
    """Batch 32 at 256x256 (the FNO throughput workload); the oracle checks two sampled items."""
    _requires_gpu()
    s, g, params = _pair(width=32, layers=4, modes=12, dec_size=32, seed=0, out_scale=1e-2)
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(256, 256)
    x = _flow_inputs(32, 256, 256)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(32, 256, 256)
    for b in (0, 31):
        ref = fo.fno_forward(s, params, x[b:b + 1])[0]
        e = rel_l2(y[b], ref)
        print(f"FNO 32x256x256 item {b}: rel L2 {e:.3e}")
        assert e < REL_L2_FNO
    # items are independent: a batch of one gives the same result
    y1 = net(torch.from_numpy(x[5:6].copy()).cuda()).cpu().numpy()
    np.testing.assert_array_equal(y1[0], y[5])


def test_fno_throughput_workload_every_item_against_oracle():
    """Batch 32 at 256x256 (the FNO throughput workload): every item element by element."""
    _requires_gpu()
    s, g, params = _pair(width=32, layers=4, modes=12, dec_size=32, seed=0, out_scale=1e-2)
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(256, 256)
    x = _flow_inputs(32, 256, 256)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(32, 256, 256)
    ref = fo.fno_forward(s, params, x)
    errs = [rel_l2(y[b], ref[b]) for b in range(32)]
    print(f"FNO 32x256x256 all items: rel L2 max {max(errs):.3e} mean {np.mean(errs):.3e}")
    assert max(errs) < REL_L2_FNO and rel_l2(y, ref) < REL_L2_FNO


def test_bench_batch_shape_on_tensor_cores():
    """The bench's steady-framework FNO (C=32, m=12, 4 layers) on its 256 x 512 porous grids,
    B = 8, input (rho-1 = 0, u = 0, mask) as the steady driver feeds it."""
    _requires_gpu()
    s, g, params = _pair(width=32, layers=4, modes=12, dec_size=32, seed=0, out_scale=1.0)
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(256, 512)
    x = np.zeros((8, 4, 256, 512), np.float32)
    for b in range(8):
        x[b, 3] = synth.porous_media(512, 256, 4, 12, seed=b)[0]
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(8, 256, 512)
    ref = fo.fno_forward(s, params, x)
    errs = [rel_l2(y[b], ref[b]) for b in range(8)]
    print(f"FNO 8x256x512 porous: rel L2 max {max(errs):.3e}")
    assert max(errs) < REL_L2_FNO


def test_spectral_chain_alone_at_full_size():
    """Fourier layers with W = 0 and b = 0 and a decoder without biases: the output is then
    carried entirely by the x-DFT, y-DFT, mixing and inverse chain of every layer, so the
    relative L2 measures that chain (B = 8 of the 256x256 throughput workload)."""
    _requires_gpu()
    s, g, params = _pair(width=32, layers=4, modes=12, dec_size=32, seed=2, out_scale=1.0)
    for n in range(4):
        params[f"layer{n}.w"] = np.zeros_like(params[f"layer{n}.w"])
        params[f"layer{n}.b"] = np.zeros_like(params[f"layer{n}.b"])
        for blk in ("r1.re", "r1.im", "r2.re", "r2.im"):  # gain O(1) per layer
            k = f"layer{n}.{blk}"
            params[k] = synth.round_to_bf16((params[k] * 128).astype(np.float32))
    params["dec0.b"] = np.zeros_like(params["dec0.b"])
    params["out.b"] = np.zeros_like(params["out.b"])
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(256, 256)
    x = _flow_inputs(8, 256, 256, seed0=40)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(8, 256, 256)
    ref = fo.fno_forward(s, params, x)
    # the chain is not trivial: outputs vary in space (not a constant field)
    assert np.std(ref[0, 0]) > 1e-3 * np.abs(ref[0, 0]).max() > 0
    errs = [rel_l2(y[b], ref[b]) for b in range(8)]
    print(f"FNO spectral chain alone 8x256x256: rel L2 max {max(errs):.3e}")
    assert max(errs) < REL_L2_FNO


def test_invalid_fno_shapes_rejected():
    _requires_gpu()
    s, g, params = _pair(modes=4)
    net = Fno(g, synth.fno_flatten_params(s, params))
    with pytest.raises(P.LbmError):
        net(torch.zeros((1, 4, 7, 16), device="cuda"))  # 2m > H
    with pytest.raises(P.LbmError):
        net(torch.zeros((1, 4, 16, 8), device="cuda"))  # m >= W/2


def test_tensor_core_activation_matches_exact_gelu():
    """The tensor-core kernels' GELU (Gaussian-tail polynomial times exp) against the exact
    v Phi(v) in FP64 (math.erf) on a dense grid, its tails, and special values."""
    _requires_gpu()
    import math
    from paper_2604_27158_gb300.fno import activation
    v = np.concatenate([np.linspace(-12.0, 12.0, 2_000_001), np.linspace(-1e-3, 1e-3, 20001),
                        [-50.0, -7.0, -6.0, 6.0, 7.0, 50.0, 1e20, -1e20]]).astype(np.float32)
    got = activation(torch.from_numpy(v).cuda()).cpu().numpy().astype(np.float64)
    vd = v.astype(np.float64)
    ref = np.array([0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0))) for x in vd.tolist()])
    err = np.abs(got - ref) / (1.0 + np.abs(vd))
    print(f"GELU: max |err| / (1 + |v|) = {err.max():.2e}")
    assert err.max() < 5e-6
    special = torch.tensor([float("nan"), float("inf"), 0.0, -0.0], device="cuda")
    out = activation(special).cpu().numpy()
    assert np.isnan(out[0]) and out[1] == np.inf and out[2] == 0.0 and out[3] == 0.0
    relu = activation(torch.from_numpy(v).cuda(), P._abi.FNO_ACT_RELU).cpu().numpy()
    np.testing.assert_array_equal(relu, np.maximum(v, 0.0))


@pytest.mark.parametrize("H,W,width,act", [(32, 128, 32, 0), (64, 256, 32, 0), (40, 128, 16, 0),
                                            (32, 128, 64, 0), (24, 128, 32, 1), (24, 256, 64, 1)])
def test_tensor_core_path_matches_oracle(H, W, width, act):
    """tcgen05 path (channel-blocked latents, DFT and 1x1 layers as MMAs) vs the FP64 oracle,
    with GELU and with ReLU (the activation is a compile-time parameter of the kernels)."""
    _requires_gpu()
    s, g, params = _pair(width=width, layers=3, modes=12 if width != 16 else 6,
                         dec_size=width, seed=11, act=act)
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(H, W)
    x = _inputs(2, 4, H, W, seed=13)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(2, H, W)
    ref = fo.fno_forward(s, params, x, activation="gelu" if act == 0 else "relu")
    e = rel_l2(y, ref)
    print(f"FNO tensor cores C={width} {H}x{W} act={act}: rel L2 {e:.3e}")
    assert e < REL_L2_FNO


def test_tensor_core_and_cuda_core_paths_agree():
    _requires_gpu()
    s, g, params = _pair(width=32, layers=4, modes=12, dec_size=32, seed=3)
    net = Fno(g, synth.fno_flatten_params(s, params))
    x = torch.from_numpy(_inputs(3, 4, 64, 128, seed=4)).cuda()
    y_tc = net(x).cpu().numpy()
    net.check(3, 64, 128)
    net.set_path(P._abi.FNO_PATH_CUDA_CORES)
    assert not net.uses_tensor_cores(64, 128)
    y_cc = net(x).cpu().numpy()
    e = rel_l2(y_tc, y_cc)
    print(f"tensor-core vs CUDA-core path: rel L2 {e:.3e}")
    assert e < REL_L2_FNO


@pytest.mark.parametrize("name,cin,cout,width,layers,modes,dec_layers,dec,B,H,W", [
    ("porous density model (114,273 params)", 1, 1, 16, 3, 6, 3, 32, 2, 64, 128),
    ("porous velocity model (896,082 params)", 1, 2, 16, 6, 12, 3, 64, 1, 64, 128),
    ("shear velocity model, 3 layers (2,409,771 params)", 2, 2, 14, 3, 32, 1, 32, 2, 64, 64),
])
def test_paper_models_with_padding_match_oracle(name, cin, cout, width, layers, modes, dec_layers,
                                                dec, B, H, W):
    """The appendix-table architectures with "Padding: 9" (latent field zero-padded after
    lifting, cropped after the last Fourier layer), on the tensor-core path (channels
    padded to 16 with zero weights, grids padded to the tile sizes, 2m up to 64 kept
    x-frequencies) and with the path forced to CUDA cores."""
    _requires_gpu()
    s = synth.FnoShape(c_in=cin, c_out=cout, width=width, layers=layers, modes=modes,
                       dec_layers=dec_layers, dec_size=dec, padding=9)
    g = FnoShape(c_in=cin, c_out=cout, width=width, layers=layers, modes=modes,
                 dec_layers=dec_layers, dec_size=dec, padding=9)
    params = synth.fno_random_params(s, seed=21, out_scale=1.0)
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(H, W)
    x = _inputs(B, cin, H, W, seed=23)
    ref = fo.fno_forward(s, params, x)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(B, H, W)
    e = rel_l2(y, ref)
    net.set_path(P._abi.FNO_PATH_CUDA_CORES)
    y_cc = net(torch.from_numpy(x).cuda()).cpu().numpy()
    e_cc = rel_l2(y_cc, ref)
    print(f"{name} padded {B}x{H}x{W}: rel L2 tensor cores {e:.3e}, CUDA cores {e_cc:.3e} "
          f"({fo.param_count(s)} params)")
    assert e < REL_L2_FNO and e_cc < REL_L2_FNO


@pytest.mark.parametrize("cin,width,act", [(1, 16, 0), (2, 32, 1), (3, 16, 0), (4, 64, 0),
                                            (7, 64, 1), (16, 32, 0)])
def test_lift_input_widths_on_tensor_cores(cin, width, act):
    """The tensor-core lift has instances for 1, 2 and 4 input channels and one with a
    runtime input width (up to 16) for the rest: each against the oracle, on grids with a
    ragged last x tile (W = 150: tiles of 128 and 22 pixels in 192-pixel storage rows)
    and more tiles than CTAs, with both activations."""
    _requires_gpu()
    s, g, params = _pair(c_in=cin, c_out=2, width=width, layers=1, modes=4, dec_size=32,
                         act=act, seed=cin + width)
    net = Fno(g, synth.fno_flatten_params(s, params))
    B, H, W = 6, 200, 150
    assert net.uses_tensor_cores(H, W)
    x = _inputs(B, cin, H, W, seed=cin)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(B, H, W)
    ref = fo.fno_forward(s, params, x, activation="gelu" if act == 0 else "relu")
    e = rel_l2(y, ref)
    print(f"lift c_in={cin} C={width} act={act} {B}x{H}x{W}: rel L2 {e:.3e}")
    assert e < REL_L2_FNO


@pytest.mark.parametrize("width,B,H,pad", [(16, 1, 37, 0), (32, 1, 37, 0), (16, 3, 29, 0),
                                           (32, 1, 28, 9)])
def test_multi_row_tiles_with_short_last_tile(width, B, H, pad):
    """The tensor-core inverse x-DFT (four rows a tile at C = 16, two at C = 32), decoder
    (two rows) and lift (two rows at C = 16) on row counts that leave a short last tile
    (B H0 or B Hv odd, or not a multiple of four), W = 128 so the decoder takes the
    tensor cores; against the oracle."""
    _requires_gpu()
    s = synth.FnoShape(c_in=4, c_out=3, width=width, layers=2, modes=5, dec_size=32,
                       padding=pad)
    g = FnoShape(c_in=4, c_out=3, width=width, layers=2, modes=5, dec_size=32, padding=pad)
    params = synth.fno_random_params(s, seed=width + H, out_scale=1.0)
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(H, 128)
    x = _inputs(B, 4, H, 128, seed=H)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(B, H, 128)
    e = rel_l2(y, fo.fno_forward(s, params, x))
    print(f"multi-row tiles C={width} {B}x{H}x128 pad {pad}: rel L2 {e:.3e}")
    assert e < REL_L2_FNO


@pytest.mark.parametrize("which", ["density", "velocity"])
def test_double_shear_model_pair_on_tensor_cores(which):
    """The 2.6 M double-shear model group (Sec. 3.2.1; 14 channels, 3 layers, decoder 32,
    padding 9) at its workload size, B = 4 periodic 128 x 128 fields -> 137 x 137 padded
    grid: density net (rho - 1 -> rho - 1, 8 modes) and velocity net ((u, v) -> (u, v),
    32 modes: 64 kept x-frequencies)."""
    _requires_gpu()
    cin, modes = (1, 8) if which == "density" else (2, 32)
    s = synth.FnoShape(c_in=cin, c_out=cin, width=14, layers=3, modes=modes, dec_size=32,
                       padding=9)
    g = FnoShape(c_in=cin, c_out=cin, width=14, layers=3, modes=modes, dec_size=32, padding=9)
    params = synth.fno_random_params(s, seed=31 if which == "density" else 32, out_scale=1.0)
    assert fo.param_count(s) == (151811 if which == "density" else 2409771)
    net = Fno(g, synth.fno_flatten_params(s, params))
    assert net.uses_tensor_cores(128, 128)
    ics = synth.double_shear(4, seed=2000)
    planes = [("rho",)] if which == "density" else [("ux",), ("uy",)]
    x = np.stack([np.stack([(ic["rho"] - 1.0) if k[0] == "rho" else ic[k[0]] for k in planes])
                  for ic in ics]).astype(np.float32)
    y = net(torch.from_numpy(x).cuda()).cpu().numpy()
    net.check(4, 128, 128)
    ref = fo.fno_forward(s, params, x)
    errs = [rel_l2(y[b], ref[b]) for b in range(4)]
    print(f"double-shear {which} net on tensor cores: rel L2 max {max(errs):.3e}")
    assert max(errs) < REL_L2_FNO
