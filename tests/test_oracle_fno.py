"""Pins of the FP64 FNO oracle (Sec. 2.2) against brute force, a library FFT,
closed-form properties and the parameter counts printed in the paper."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import fno_oracle as fo
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("H,W,m", [(8, 8, 3), (8, 12, 4), (6, 10, 2)])
def test_truncated_dft_matches_brute_force_double_sum(H, W, m):
    rng = np.random.default_rng(H * 100 + W)
    th = rng.standard_normal((H, W))
    X = fo.truncated_dft(th, m)
    kys = list(range(m)) + list(range(H - m, H))
    for a, ky in enumerate(kys):
        for kx in range(m):
            s = 0j
            for y in range(H):
                for x in range(W):
                    s += th[y, x] * complex(math.cos(-2 * math.pi * (ky * y / H + kx * x / W)),
                                            math.sin(-2 * math.pi * (ky * y / H + kx * x / W)))
            assert abs(X[a, kx] - s) < 1e-12


def test_truncated_idft_matches_brute_force_double_sum():
    H, W, m = 8, 10, 3
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((2 * m, m)) + 1j * rng.standard_normal((2 * m, m))
    s = fo.truncated_idft(Y, H, W)
    kys = list(range(m)) + list(range(H - m, H))
    for y in range(H):
        for x in range(W):
            acc = 0.0
            for a, ky in enumerate(kys):
                for kx in range(m):
                    c = 1.0 if kx == 0 else 2.0
                    ph = 2 * math.pi * (ky * y / H + kx * x / W)
                    acc += c * (Y[a, kx] * complex(math.cos(ph), math.sin(ph))).real
            assert abs(s[y, x] - acc / (H * W)) < 1e-13


@pytest.mark.parametrize("H,W,m", [(16, 16, 5), (12, 20, 6), (32, 16, 7)])
def test_spectral_conv_matches_library_rfft2_pipeline(H, W, m):
    # the library realisation: rfft2 -> keep the two corner blocks -> mix -> irfft2
    rng = np.random.default_rng(7)
    B, Ci, Co = 2, 3, 4
    th = rng.standard_normal((B, Ci, H, W))
    r1 = rng.standard_normal((Ci, Co, m, m)) + 1j * rng.standard_normal((Ci, Co, m, m))
    r2 = rng.standard_normal((Ci, Co, m, m)) + 1j * rng.standard_normal((Ci, Co, m, m))
    ours = fo.spectral_conv(th, r1, r2)
    t = torch.from_numpy(th)
    xf = torch.fft.rfft2(t)
    out = torch.zeros(B, Co, H, W // 2 + 1, dtype=torch.complex128)
    out[:, :, :m, :m] = torch.einsum("bixy,ioxy->boxy", xf[:, :, :m, :m], torch.from_numpy(r1))
    out[:, :, -m:, :m] = torch.einsum("bixy,ioxy->boxy", xf[:, :, -m:, :m], torch.from_numpy(r2))
    ref = torch.fft.irfft2(out, s=(H, W)).numpy()
    np.testing.assert_allclose(ours, ref, atol=1e-12)


def test_identity_filter_passes_kept_modes_and_halves_the_unpaired_one():
    # With R = 1 the spectral convolution keeps every real Fourier component whose
    # modes (ky, kx) and (-ky, -kx) are both retained, removes the others, and -
    # because the kx = 0 column keeps ky = H - m but not its partner ky = m -
    # passes cos(2 pi m y / H) with weight 1/2 (Hermitian half-spectrum inverse).
    H, W, m = 16, 12, 4
    one = np.ones((1, 1, m, m), dtype=np.complex128)
    y = np.arange(H)[:, None] * np.ones((1, W))
    x = np.arange(W)[None, :] * np.ones((H, 1))
    band = (np.cos(2 * np.pi * (2 * y / H + 1 * x / W)) + 0.5 * np.sin(2 * np.pi * (3 * x / W - 1 * y / H))
            + 0.25 + 0.3 * np.cos(2 * np.pi * 3 * y / H))
    np.testing.assert_allclose(fo.spectral_conv(band[None, None], one, one)[0, 0], band, atol=1e-12)
    cut = np.cos(2 * np.pi * (5 * y / H)) + np.sin(2 * np.pi * (4 * x / W))  # outside the kept set
    np.testing.assert_allclose(fo.spectral_conv(cut[None, None], one, one)[0, 0], 0.0, atol=1e-12)
    unpaired = np.cos(2 * np.pi * m * y / H)
    np.testing.assert_allclose(fo.spectral_conv(unpaired[None, None], one, one)[0, 0], 0.5 * unpaired,
                               atol=1e-12)


def test_gelu_textbook_values():
    x = np.array([0.0, 1.0, -1.0, 2.0])
    # Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208 (standard normal CDF)
    ref = np.array([0.0, 0.8413447460685429, -1 + 0.8413447460685429, 2 * 0.9772498680518208])
    np.testing.assert_allclose(fo.gelu(x), ref, atol=1e-15)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 10,
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -3.0e-5, 65504.0], np.float32)])
    ours = fo.bf16(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)
    np.testing.assert_array_equal(synth.round_to_bf16(v).astype(np.float64), ref)


def test_parameter_counts_match_paper_tables():
    with open(os.path.join(GOLDEN, "fno_param_counts.json")) as fh:
        gold = json.load(fh)
    counts = {}
    for mdl in gold["models"]:
        shape = synth.FnoShape(c_in=mdl["c_in"], c_out=mdl["c_out"], width=mdl["width"],
                               layers=mdl["layers"], modes=mdl["modes"],
                               dec_layers=mdl["dec_layers"], dec_size=mdl["dec_size"])
        counts[mdl["name"]] = fo.param_count(shape)
        assert counts[mdl["name"]] == mdl["params"], mdl["name"]
    names = [m["name"] for m in gold["models"]]
    assert counts[names[3]] + counts[names[5]] == gold["group_totals"]["11.2M FNO"]
    assert counts[names[2]] + counts[names[4]] == gold["group_totals"]["2.6M FNO"]


def test_hot_path_fno_size_is_about_2_5M():
    # 4 layers, 32 latent channels, 12x12 modes, (rho, ux, uy, mask) -> 3 fields
    n = fo.param_count(synth.FnoShape())
    assert n == 2365331


def _torch_fno(shape, params, phi, act):
    """Independent float64 torch realisation (conv1x1 + rfft2/irfft2), PhysicsNeMo-style."""
    p = {k: torch.from_numpy(fo.bf16(v)) for k, v in params.items()}
    x = torch.from_numpy(fo.bf16(phi))
    B, _, H, W = x.shape
    gx = torch.linspace(0, 1, W, dtype=torch.float64)
    gy = torch.linspace(0, 1, H, dtype=torch.float64)
    gyy, gxx = torch.meshgrid(gy, gx, indexing="ij")
    coords = torch.from_numpy(fo.bf16(torch.stack([gxx, gyy]).numpy().astype(np.float32)))
    x = torch.cat([x, coords[None].expand(B, -1, -1, -1)], 1)
    a = torch.nn.functional.gelu if act == "gelu" else torch.relu
    conv = lambda w, b, t: torch.nn.functional.conv2d(t, w[:, :, None, None], b)
    h = conv(p["lift1.w"], p["lift1.b"], a(conv(p["lift0.w"], p["lift0.b"], x)))
    m = shape.modes
    for n in range(shape.layers):
        r1 = torch.complex(p[f"layer{n}.r1.re"], p[f"layer{n}.r1.im"])
        r2 = torch.complex(p[f"layer{n}.r2.re"], p[f"layer{n}.r2.im"])
        xf = torch.fft.rfft2(h)
        of = torch.zeros(B, shape.width, H, W // 2 + 1, dtype=torch.complex128)
        of[:, :, :m, :m] = torch.einsum("bixy,ioxy->boxy", xf[:, :, :m, :m], r1)
        of[:, :, -m:, :m] = torch.einsum("bixy,ioxy->boxy", xf[:, :, -m:, :m], r2)
        h = a(conv(p[f"layer{n}.w"], p[f"layer{n}.b"], h) + torch.fft.irfft2(of, s=(H, W)))
    for l in range(shape.dec_layers):
        h = a(conv(p[f"dec{l}.w"], p[f"dec{l}.b"], h))
    return conv(p["out.w"], p["out.b"], h).numpy()


@pytest.mark.parametrize("act", ["gelu", "relu"])
def test_fno_forward_matches_library_realisation(act):
    shape = synth.FnoShape(c_in=4, c_out=3, width=8, layers=2, modes=3, dec_layers=1, dec_size=8)
    params = synth.fno_random_params(shape, seed=1, out_scale=1.0)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((2, 4, 12, 16)).astype(np.float32)
    ours = fo.fno_forward(shape, params, phi, activation=act)
    ref = _torch_fno(shape, params, phi, act)
    np.testing.assert_allclose(ours, ref, atol=1e-11, rtol=1e-11)


def test_fno_without_spectral_part_is_pointwise():
    # with R = 0 every output pixel depends only on its own input pixel
    shape = synth.FnoShape(c_in=4, c_out=3, width=8, layers=2, modes=3, dec_layers=1, dec_size=8)
    params = synth.fno_random_params(shape, seed=2, out_scale=1.0)
    for k in params:
        if ".r1." in k or ".r2." in k:
            params[k] = np.zeros_like(params[k])
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((1, 4, 8, 8)).astype(np.float32)
    out = fo.fno_forward(shape, params, phi)
    phi2 = phi.copy()
    phi2[0, :, 3, 5] += 1.0
    out2 = fo.fno_forward(shape, params, phi2)
    diff = np.abs(out2 - out).sum(axis=(0, 1))
    assert diff[3, 5] > 0 and np.count_nonzero(diff > 1e-14) == 1


def test_padding_with_zero_spectral_filters_is_invisible():
    """With all spectral filters zero the network is pointwise, so padding the latent field
    and cropping it back must not change the output (a crop of the wrong corner would:
    the padded cells hold sigma(b), not the interior values)."""
    base = synth.FnoShape(width=8, layers=2, modes=3, dec_size=8)
    padded = synth.FnoShape(width=8, layers=2, modes=3, dec_size=8, padding=5)
    params = synth.fno_random_params(base, seed=3, out_scale=1.0)
    for n in range(2):
        for k in ("r1.re", "r1.im", "r2.re", "r2.im"):
            params[f"layer{n}.{k}"] = np.zeros_like(params[f"layer{n}.{k}"])
    x = np.random.default_rng(1).standard_normal((2, 4, 9, 11))
    np.testing.assert_allclose(fo.fno_forward(padded, params, x), fo.fno_forward(base, params, x),
                               rtol=0, atol=1e-13)


def test_padded_layer_matches_brute_force_sums():
    """One padded Fourier layer written out with explicit loops: zero-extend the lifted field
    to (H+p) x (W+p), truncated DFT / mixing / Hermitian inverse as double sums over the
    padded grid, + W theta + b, GELU, crop to H x W, decoder."""
    shape = synth.FnoShape(c_in=1, c_out=1, width=2, layers=1, modes=2, dec_size=2, padding=3)
    params = synth.fno_random_params(shape, seed=5, out_scale=1.0)
    p = {k: fo.bf16(v) for k, v in params.items()}
    H, W, pad = 4, 5, 3
    x = fo.bf16(np.random.default_rng(2).standard_normal((1, 1, H, W)))
    Hp, Wp, m, C = H + pad, W + pad, 2, 2
    coords = fo.coordinate_channels(H, W)
    theta = np.zeros((C, Hp, Wp))
    for y in range(H):
        for xx in range(W):
            v = np.array([x[0, 0, y, xx], coords[0, y, xx], coords[1, y, xx]])
            h = fo.gelu(p["lift0.w"] @ v + p["lift0.b"])
            theta[:, y, xx] = p["lift1.w"] @ h + p["lift1.b"]
    kys = list(range(m)) + list(range(Hp - m, Hp))
    R = np.concatenate([p["layer0.r1.re"] + 1j * p["layer0.r1.im"],
                        p["layer0.r2.re"] + 1j * p["layer0.r2.im"]], axis=2)  # [i][o][a][kx]
    Xh = np.zeros((C, 2 * m, m), complex)
    for i in range(C):
        for a, ky in enumerate(kys):
            for kx in range(m):
                Xh[i, a, kx] = sum(theta[i, y, xx] * np.exp(-2j * np.pi * (ky * y / Hp + kx * xx / Wp))
                                   for y in range(Hp) for xx in range(Wp))
    Yh = np.einsum("iak,ioak->oak", Xh, R)
    out = np.zeros((C, Hp, Wp))
    for o in range(C):
        for y in range(Hp):
            for xx in range(Wp):
                s = 0.0
                for a, ky in enumerate(kys):
                    for kx in range(m):
                        s += (1.0 if kx == 0 else 2.0) * np.real(
                            Yh[o, a, kx] * np.exp(2j * np.pi * (ky * y / Hp + kx * xx / Wp)))
                lin = p["layer0.w"][o] @ theta[:, y, xx] + p["layer0.b"][o]
                out[o, y, xx] = fo.gelu(lin + s / (Hp * Wp))
    ref = np.zeros((1, 1, H, W))
    for y in range(H):
        for xx in range(W):
            h = fo.gelu(p["dec0.w"] @ out[:, y, xx] + p["dec0.b"])
            ref[0, 0, y, xx] = (p["out.w"] @ h + p["out.b"])[0]
    np.testing.assert_allclose(fo.fno_forward(shape, params, x), ref, rtol=0, atol=1e-12)

