"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *draws* inputs: obstacle geometries, macroscopic fields, FNO
parameters.  It holds none of the method's arithmetic (no equilibrium, no
collision, no streaming, no DFT); both the FP64 oracle and the CUDA path take
what it returns as plain arrays.

Geometry follows the paper's workloads:
  * porous media (Sec. 3.1.1): a rectangular channel, periodic sides, inlet and
    outlet columns, populated with non-overlapping random disks until the
    porosity phi = 1 - A_solid / A_total (Eq. for phi in Sec. 3.1.1) reaches a
    drawn target;
  * a periodic-in-x channel with solid wall rows and a few disks (the plain LBM
    workload), and the flow-past-disks grids of the batched hybrid workload.

Disk rasterisation is integer-exact: cell (x, y) is solid iff
(x - cx)^2 + (y - cy)^2 <= r^2 in integers, with the minimum-image distance in
periodic dimensions.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "Disk",
    "rasterise_disks",
    "channel_with_disks",
    "porous_media",
    "flow_past_disks",
    "pack_mask_bits",
    "round_to_bf16",
    "FnoShape",
    "fno_param_shapes",
    "fno_random_params",
    "fno_flatten_params",
    "smooth_macro_fields",
    "DoubleShear",
    "double_shear",
    "unsteady_batch",
    "random_post_collision_state",
]


@dataclasses.dataclass(frozen=True)
class Disk:
    cx: int
    cy: int
    r: int


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _wrap_delta(d: np.ndarray, n: int, periodic: bool) -> np.ndarray:
    if not periodic:
        return d
    d = np.mod(d, n)
    return np.minimum(d, n - d)


def rasterise_disks(nx: int, ny: int, disks: Sequence[Disk], periodic_x: bool,
                    periodic_y: bool) -> np.ndarray:
    """Boolean solid mask [ny, nx] (True = solid) of integer disks."""
    solid = np.zeros((ny, nx), dtype=bool)
    xs = np.arange(nx, dtype=np.int64)[None, :]
    ys = np.arange(ny, dtype=np.int64)[:, None]
    for d in disks:
        dx = _wrap_delta(xs - d.cx, nx, periodic_x)
        dy = _wrap_delta(ys - d.cy, ny, periodic_y)
        solid |= (dx * dx + dy * dy) <= d.r * d.r
    return solid


def _center_dist2(a: Disk, cx: int, cy: int, nx: int, ny: int, px: bool, py: bool) -> int:
    dx = abs(a.cx - cx)
    dy = abs(a.cy - cy)
    if px:
        dx = min(dx, nx - dx)
    if py:
        dy = min(dy, ny - dy)
    return dx * dx + dy * dy


def _place_disks(rng, nx, ny, px, py, rmin, rmax, x_range, y_range, gap, stop, max_tries=200000):
    disks: List[Disk] = []
    tries = 0
    while not stop(disks) and tries < max_tries:
        tries += 1
        r = int(rng.integers(rmin, rmax + 1))
        xlo, xhi = x_range(r)
        ylo, yhi = y_range(r)
        if xhi < xlo or yhi < ylo:
            continue
        cx = int(rng.integers(xlo, xhi + 1))
        cy = int(rng.integers(ylo, yhi + 1))
        ok = True
        for d in disks:
            need = d.r + r + gap
            if _center_dist2(d, cx, cy, nx, ny, px, py) < need * need:
                ok = False
                break
        if ok:
            disks.append(Disk(cx, cy, r))
    return disks


def channel_with_disks(nx: int = 128, ny: int = 64, ndisks: int = 6, rmin: int = 4,
                       rmax: int = 8, seed: int = 0) -> Tuple[np.ndarray, List[Disk]]:
    """Periodic-in-x channel: solid wall rows y=0 and y=ny-1, plus `ndisks` disks.

    Disks do not overlap each other (gap >= 2 cells) nor touch the walls.
    Returns (solid[ny, nx] bool, disks).
    """
    rng = _rng(seed)
    disks = _place_disks(
        rng, nx, ny, True, False, rmin, rmax,
        x_range=lambda r: (0, nx - 1),
        y_range=lambda r: (r + 2, ny - 3 - r),
        gap=2, stop=lambda ds: len(ds) >= ndisks)
    solid = rasterise_disks(nx, ny, disks, periodic_x=True, periodic_y=False)
    solid[0, :] = True
    solid[ny - 1, :] = True
    return solid, disks


def porous_media(nx: int = 512, ny: int = 256, rmin: int = 4, rmax: int = 12,
                 porosity_range: Tuple[float, float] = (0.6, 0.8), seed: int = 0,
                 gap: int = 2) -> Tuple[np.ndarray, List[Disk], float]:
    """Porous medium: periodic in y, inlet column x=0 and outlet column x=nx-1.

    A porosity target phi* ~ U(porosity_range) is drawn; non-overlapping disks
    (centre distance >= r1 + r2 + gap, with the periodic minimum image in y) are
    added by random sequential placement until the porosity of the rasterised
    mask is <= phi*, or placement saturates.  Disk centres keep >= r + 2 cells
    from the inlet and outlet columns.  Returns (solid, disks, achieved phi).
    """
    rng = _rng(seed)
    target = float(rng.uniform(*porosity_range))
    total = nx * ny
    # disk areas in integer cells, cached per radius
    area = {}
    for r in range(rmin, rmax + 1):
        d = np.arange(-r, r + 1)
        area[r] = int(((d[:, None] ** 2 + d[None, :] ** 2) <= r * r).sum())
    solid_cells = [0]

    def stop(ds):
        if ds:
            # disks never overlap, so the solid area is the sum of disk areas
            solid_cells[0] = sum(area[d.r] for d in ds)
        return 1.0 - solid_cells[0] / total <= target

    disks = _place_disks(
        rng, nx, ny, False, True, rmin, rmax,
        x_range=lambda r: (r + 2, nx - 1 - (r + 2)),
        y_range=lambda r: (0, ny - 1),
        gap=gap, stop=stop)
    solid = rasterise_disks(nx, ny, disks, periodic_x=False, periodic_y=True)
    phi = 1.0 - solid.sum() / total
    return solid, disks, float(phi)


def flow_past_disks(nx: int, ny: int, seed: int, ndisks_range=(1, 4),
                    rmin: int = 4, rmax: int = 16) -> Tuple[np.ndarray, List[Disk]]:
    """Flow past 1-4 random disks in a periodic-in-y channel with inlet/outlet columns.

    Disks sit in the middle 60% of the channel length and do not overlap.
    """
    rng = _rng(seed)
    n = int(rng.integers(ndisks_range[0], ndisks_range[1] + 1))
    rmax_eff = max(rmin, min(rmax, ny // 8))
    disks = _place_disks(
        rng, nx, ny, False, True, rmin, rmax_eff,
        x_range=lambda r: (int(0.2 * nx) + r, int(0.8 * nx) - r),
        y_range=lambda r: (0, ny - 1),
        gap=2, stop=lambda ds: len(ds) >= n)
    solid = rasterise_disks(nx, ny, disks, periodic_x=False, periodic_y=True)
    return solid, disks


UNSTEADY_SIZES = ((128, 128), (256, 128), (256, 256), (512, 256))  # (nx, ny)


def unsteady_batch(n: int, seed: int = 0, sizes=UNSTEADY_SIZES, tau_range=(0.55, 0.8),
                   re_range=(50.0, 200.0), u_cap: float = 0.08):
    """Batch of flow-past-disks trajectories of uneven size (the super-time-stepping workload).

    Per trajectory: a size drawn from `sizes`, 1-4 disks (flow_past_disks), tau ~
    U(tau_range), a Reynolds number Re ~ U(re_range) based on the channel height
    ny, and the inlet speed U = Re nu / ny with nu = (tau - 1/2) / 3, capped at
    `u_cap` for Mach safety (the effective Re is returned).  Velocity inlet,
    pressure outlet rho = 1, periodic in y.
    Returns a list of dicts {nx, ny, tau, u_in, re, solid}.
    """
    rng = _rng(seed)
    out = []
    for k in range(n):
        nx, ny = sizes[int(rng.integers(0, len(sizes)))]
        tau = float(rng.uniform(*tau_range))
        re = float(rng.uniform(*re_range))
        solid, _ = flow_past_disks(nx, ny, seed=int(rng.integers(0, 2 ** 31)))
        nu = (tau - 0.5) / 3.0
        u = min(re * nu / ny, u_cap)
        out.append(dict(nx=nx, ny=ny, tau=tau, u_in=u, re=u * ny / nu, solid=solid))
    return out


@dataclasses.dataclass(frozen=True)
class DoubleShear:
    """Lattice set-up of the double-shear-layer workload (Sec. 3.2.1): a periodic unit
    square at n x n cells, U = 1 m/s, nu = 1e-3 m^2/s, and an FNO time step of
    Delta T = 0.1 s = 223 LBM steps (30 Delta T = 3 s of simulated time)."""
    n: int = 128
    steps_per_dT: int = 223
    dT_seconds: float = 0.1
    U: float = 1.0
    nu: float = 1e-3

    @property
    def dt(self) -> float:  # seconds per LBM step
        return self.dT_seconds / self.steps_per_dT

    @property
    def u_lattice(self) -> float:  # lattice velocity of U
        return self.U * self.dt * self.n

    @property
    def tau(self) -> float:  # 1/2 + 3 nu dt / dx^2
        return 0.5 + 3.0 * self.nu * self.dt * self.n * self.n


def double_shear(count: int, seed: int = 0, setup: DoubleShear = DoubleShear(),
                 a_range=(20.0, 125.0), upper=(0.65, 0.85), lower=(0.15, 0.35)):
    """Initial conditions of the double shear layer in lattice units.

    u = U tanh(A1 (x2' - x2)) for x2 >= 0.5 and U tanh(A2 (x2 - x2'')) for x2 < 0.5,
    v = 0.1 U sin(2 pi (x1 + 1/4)), on cell centres x = (i + 1/2)/n.  A1, A2 are drawn
    from a_range (Re = U delta / nu with delta = 1/A spans 8 .. 50), the layer centres
    x2' and x2'' from `upper` and `lower`.  Returns one dict per trajectory with rho, ux,
    uy ([n, n] float32, rho = 1) and the drawn parameters.
    """
    rng = _rng(seed)
    n = setup.n
    c = (np.arange(n) + 0.5) / n
    x1 = c[None, :]
    x2 = c[:, None]
    out = []
    for _ in range(count):
        a1, a2 = (float(v) for v in rng.uniform(*a_range, size=2))
        y_up, y_lo = float(rng.uniform(*upper)), float(rng.uniform(*lower))
        u = np.where(x2 >= 0.5, np.tanh(a1 * (y_up - x2)), np.tanh(a2 * (x2 - y_lo)))
        u = np.broadcast_to(u, (n, n))
        v = np.broadcast_to(0.1 * np.sin(2.0 * np.pi * (x1 + 0.25)), (n, n))
        ul = setup.u_lattice
        out.append({"rho": np.ones((n, n), np.float32), "ux": (ul * u).astype(np.float32),
                    "uy": (ul * v).astype(np.float32), "A1": a1, "A2": a2, "x2_upper": y_up,
                    "x2_lower": y_lo})
    return out


def pack_mask_bits(solid: np.ndarray) -> np.ndarray:
    """Bit-pack a [ny, nx] bool mask into uint32 words, one run of ceil(nx/32) words per row.

    Bit (x % 32) of word (y * words_per_row + x // 32) is 1 iff cell (x, y) is solid.
    """
    ny, nx = solid.shape
    wpr = (nx + 31) // 32
    padded = np.zeros((ny, wpr * 32), dtype=np.uint64)
    padded[:, :nx] = solid.astype(np.uint64)
    bits = padded.reshape(ny, wpr, 32)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))[None, None, :]
    words = (bits * weights).sum(axis=2).astype(np.uint32)
    return words.reshape(-1)


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 value (ties to even); returns float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    rounded = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = rounded.astype(np.uint32)
    nan = np.isnan(a)
    out = np.where(nan, np.uint32(0x7FC00000), out)
    return out.view(np.float32).reshape(a.shape)


@dataclasses.dataclass(frozen=True)
class FnoShape:
    """Architecture of an FNO (Sec. 2.2; the appendix tables give the paper's instances).

    c_in: physical input channels (2 coordinate channels are appended);
    width: latent channels C; layers: Fourier layers N; modes: m, kept modes per
    corner block; dec_layers / dec_size: hidden layers and width of the decoder Q;
    c_out: output channels; padding: zero padding of the latent field (architecture
    option of the appendix tables; it adds no parameters).
    """
    c_in: int = 4
    c_out: int = 3
    width: int = 32
    layers: int = 4
    modes: int = 12
    dec_layers: int = 1
    dec_size: int = 32
    padding: int = 0


def fno_param_shapes(s: FnoShape):
    """Ordered (name, shape) list of every FNO parameter, in the packed order."""
    C, h = s.width, s.width // 2
    out = [("lift0.w", (h, s.c_in + 2)), ("lift0.b", (h,)),
           ("lift1.w", (C, h)), ("lift1.b", (C,))]
    for n in range(s.layers):
        for blk in ("r1", "r2"):
            out.append((f"layer{n}.{blk}.re", (C, C, s.modes, s.modes)))
            out.append((f"layer{n}.{blk}.im", (C, C, s.modes, s.modes)))
        out.append((f"layer{n}.w", (C, C)))
        out.append((f"layer{n}.b", (C,)))
    fan = C
    for l in range(s.dec_layers):
        out.append((f"dec{l}.w", (s.dec_size, fan)))
        out.append((f"dec{l}.b", (s.dec_size,)))
        fan = s.dec_size
    out.append(("out.w", (s.c_out, fan)))
    out.append(("out.b", (s.c_out,)))
    return out


def fno_random_params(s: FnoShape, seed: int = 0, out_scale: float = 1e-2):
    """Seeded random FNO parameters, rounded to bfloat16 values (held as float32).

    Pointwise layers: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases.
    Spectral filters: real and imaginary parts U[0, 1/(C*C)).
    The output layer is scaled by `out_scale` so untrained predictions are
    small perturbations.
    """
    rng = _rng(seed)
    params = {}
    for name, shape in fno_param_shapes(s):
        if ".r1." in name or ".r2." in name:
            v = rng.uniform(0.0, 1.0 / (s.width * s.width), size=shape)
        else:
            fan_in = shape[1] if len(shape) == 2 else None
            if fan_in is None:  # bias: fan_in of the matching weight
                wname = name[:-2] + ".w"
                fan_in = dict(fno_param_shapes(s))[wname][1]
            bound = 1.0 / math.sqrt(fan_in)
            v = rng.uniform(-bound, bound, size=shape)
            if name.startswith("out."):
                v = v * out_scale
        params[name] = round_to_bf16(v.astype(np.float32))
    return params


def fno_flatten_params(s: FnoShape, params) -> np.ndarray:
    """Concatenate the parameters in packed order into one float32 vector."""
    return np.concatenate([np.asarray(params[n], np.float32).reshape(-1)
                           for n, _ in fno_param_shapes(s)])


def smooth_macro_fields(nx: int, ny: int, seed: int, drho: float = 1e-2,
                        umax: float = 0.05, nwaves: int = 3):
    """Smooth periodic random (rho, ux, uy) fields [ny, nx] as float32."""
    rng = _rng(seed)
    xs = np.arange(nx)[None, :] / nx
    ys = np.arange(ny)[:, None] / ny
    fields = []
    for amp, base in ((drho, 1.0), (umax, 0.0), (umax, 0.0)):
        f = np.zeros((ny, nx))
        for _ in range(nwaves):
            kx = int(rng.integers(0, 4))
            ky = int(rng.integers(0, 4))
            ph = rng.uniform(0, 2 * np.pi)
            f += np.cos(2 * np.pi * (kx * xs + ky * ys) + ph)
        fields.append((base + amp * f / nwaves).astype(np.float32))
    return tuple(fields)


def random_post_collision_state(nx: int, ny: int, seed: int, scale: float = 1e-3) -> np.ndarray:
    """Random shifted populations g_i = f_i - w_i, shape [9, ny, nx] float32."""
    rng = _rng(seed)
    return (scale * rng.standard_normal((9, ny, nx))).astype(np.float32)
