"""FP64 reference ("oracle") of the Fourier Neural Operator of Sec. 2.2.

TEST INFRASTRUCTURE ONLY: a plain, slow restatement of the FNO forward pass in
float64 numpy.  It shares no code with the CUDA path; only the tests, the smoke
check and the benchmark's CPU-baseline leg use it.

Forward pass (Sec. 2.2, Fig. 2):
  theta_0 = P(phi)                                          lifting network
  theta_{n+1} = sigma( W theta_n + F^-1( R(k) . F(theta_n)(k) ) ),  n = 0..N-1
  phi_out = Q(theta_N)                                      projection / decoder

Readings of points the paper leaves open:
  * P is a 1x1 two-layer network (c_in + 2) -> C/2 -> C with the activation in
    between; the 2 extra input channels are coordinate grids x/(W-1), y/(H-1).
    The parameter count of the appendix tables and Sec. 3.2.1 fixes these
    shapes (see `param_count`).
  * F keeps ky in [0, m) U [H-m, H) and kx in [0, m): the unnormalised forward
    DFT  X[ky, kx] = sum_y sum_x theta(y, x) exp(-2 pi i (ky y / H + kx x / W)).
    R holds one complex [C_in, C_out, m, m] block for each ky half.
  * F^-1 is the inverse of the real-input transform pair:
    s(y, x) = (1 / (H W)) Re sum_ky sum_kx c_kx Y[ky, kx] exp(+2 pi i (ky y / H + kx x / W))
    with c_0 = 1, c_kx = 2 (kx > 0): the Hermitian half-spectrum convention.
  * sigma is applied after every Fourier layer, as the layer equation writes it.
    The paper names ReLU; the hot-path workloads use GELU (exact erf form).
    Both are available.
  * Q is `dec_layers` hidden pointwise layers of width `dec_size` with the
    activation, then a linear output layer.
  * Padding ("Padding: 9" in the appendix tables): the lifted latent field is
    zero-padded by `padding` cells at the high end of both axes, the Fourier layers
    run on the padded grid, and the field is cropped back to H x W before Q.
  * Precision: parameters and inputs are rounded to bfloat16 first, then every
    operation runs in float64, so a comparison measures only compute error.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf as _erf

from synth import FnoShape, fno_param_shapes

__all__ = ["bf16", "gelu", "relu", "dft_matrices", "truncated_dft", "truncated_idft",
           "spectral_conv", "fno_forward", "param_count", "coordinate_channels"]


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64).reshape(a32.shape)


def gelu(x: np.ndarray) -> np.ndarray:
    """GELU, exact form x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2))."""
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def relu(x: np.ndarray) -> np.ndarray:
    return np.maximum(x, 0.0)


def kept_ky(H: int, m: int) -> np.ndarray:
    return np.concatenate([np.arange(m), np.arange(H - m, H)])


def _twiddle(k: np.ndarray, n: np.ndarray, N: int, sign: float) -> np.ndarray:
    """exp(sign 2 pi i k n / N) with the phase reduced (k n mod N) before scaling."""
    ph = np.mod(np.outer(k, n), N).astype(np.float64)
    ang = sign * 2.0 * math.pi * ph / N
    return np.cos(ang) + 1j * np.sin(ang)


def dft_matrices(H: int, W: int, m: int):
    """Forward factors Fy [2m, H], Fx [W, m] and inverse factors Gy [H, 2m], Gx [m, W]."""
    ky = kept_ky(H, m)
    kx = np.arange(m)
    Fy = _twiddle(ky, np.arange(H), H, -1.0)
    Fx = _twiddle(np.arange(W), kx, W, -1.0)
    Gy = _twiddle(np.arange(H), ky, H, +1.0)
    ckx = np.where(kx == 0, 1.0, 2.0)
    Gx = ckx[:, None] * _twiddle(kx, np.arange(W), W, +1.0)
    return Fy, Fx, Gy, Gx


def truncated_dft(theta: np.ndarray, m: int) -> np.ndarray:
    """X[..., ky, kx] over the kept modes of theta[..., H, W] (matrix form of the definition)."""
    H, W = theta.shape[-2:]
    Fy, Fx, _, _ = dft_matrices(H, W, m)
    return Fy @ theta.astype(np.complex128) @ Fx


def truncated_idft(Y: np.ndarray, H: int, W: int) -> np.ndarray:
    """s[..., H, W] from the kept-mode coefficients Y[..., 2m, m]."""
    m = Y.shape[-1]
    _, _, Gy, Gx = dft_matrices(H, W, m)
    return np.real(Gy @ Y @ Gx) / (H * W)


def spectral_conv(theta: np.ndarray, r1: np.ndarray, r2: np.ndarray) -> np.ndarray:
    """F^-1(R . F(theta)) for theta [B, C_in, H, W]; r1, r2 complex [C_in, C_out, m, m]."""
    H, W = theta.shape[-2:]
    m = r1.shape[-1]
    X = truncated_dft(theta, m)                    # [B, Ci, 2m, m]
    R = np.concatenate([r1, r2], axis=2)           # [Ci, Co, 2m, m]
    Y = np.einsum("bikl,iokl->bokl", X, R)         # per-mode channel mixing
    return truncated_idft(Y, H, W)


def coordinate_channels(H: int, W: int) -> np.ndarray:
    """[2, H, W]: x / (W - 1) and y / (H - 1), bfloat16-rounded."""
    gx = np.broadcast_to(np.arange(W, dtype=np.float64)[None, :] / max(W - 1, 1), (H, W))
    gy = np.broadcast_to(np.arange(H, dtype=np.float64)[:, None] / max(H - 1, 1), (H, W))
    return bf16(np.stack([gx, gy]).astype(np.float32))


def _pointwise(wt: np.ndarray, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """1x1 convolution: out[b, o, h, w] = sum_i wt[o, i] x[b, i, h, w] + b[o]."""
    return np.einsum("oi,bihw->bohw", wt, x) + b[None, :, None, None]


def fno_forward(shape: FnoShape, params: dict, phi: np.ndarray, activation: str = "gelu",
                return_latents: bool = False):
    """FNO forward pass on phi [B, c_in, H, W]; returns [B, c_out, H, W] float64."""
    act = gelu if activation == "gelu" else relu
    p = {k: bf16(v) for k, v in params.items()}
    x = bf16(phi)
    B, _, H, W = x.shape
    coords = np.broadcast_to(coordinate_channels(H, W)[None], (B, 2, H, W))
    x = np.concatenate([x, coords], axis=1)
    # lifting network P
    h = act(_pointwise(p["lift0.w"], p["lift0.b"], x))
    theta = _pointwise(p["lift1.w"], p["lift1.b"], h)
    # optional zero padding of the latent field at the high end of both axes
    pad = getattr(shape, "padding", 0)
    if pad:
        theta = np.pad(theta, ((0, 0), (0, 0), (0, pad), (0, pad)))
    latents = [theta]
    # Fourier layers
    for n in range(shape.layers):
        r1 = p[f"layer{n}.r1.re"] + 1j * p[f"layer{n}.r1.im"]
        r2 = p[f"layer{n}.r2.re"] + 1j * p[f"layer{n}.r2.im"]
        s = spectral_conv(theta, r1, r2)
        theta = act(_pointwise(p[f"layer{n}.w"], p[f"layer{n}.b"], theta) + s)
        latents.append(theta)
    # crop back to the input grid after the last Fourier layer, then projection Q
    h = theta[:, :, :H, :W]
    for l in range(shape.dec_layers):
        h = act(_pointwise(p[f"dec{l}.w"], p[f"dec{l}.b"], h))
    out = _pointwise(p["out.w"], p["out.b"], h)
    if return_latents:
        return out, latents
    return out


def param_count(shape: FnoShape) -> int:
    """Number of trainable parameters of the architecture (sum over the packed shapes)."""
    return int(sum(int(np.prod(s)) for _, s in fno_param_shapes(shape)))
