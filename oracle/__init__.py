"""FP64 CPU oracle of the hybrid FNO-LBM hot path (arXiv 2604.27158).

TEST INFRASTRUCTURE ONLY.  Only the test suite, `__graft_entry__.smoke()` and
the CPU-baseline / reference legs of `bench.py` may import this package.  The
product path (package `paper_2604_27158_gb300`) never imports it and has no CPU
fallback.

Contents:
  * `lbm_oracle.c` (built to `liblbm_oracle.so` with gcc): D2Q9 SRT LBM,
    Sec. 2.1 — equilibrium, collision, streaming with halfway bounce-back,
    Zou-He inlet/outlet completion, moments, Guo body force, and the
    re-initialisation from macroscopic fields of the hybrid framework (Sec. 2.3).
  * `fno_oracle.py`: the FNO forward pass of Sec. 2.2 with a naive truncated DFT.
  * this module: ctypes bindings, the steady-state residual and the two hybrid
    drivers of Sec. 2.3 (FNO initialisation for steady flows, FNO/LBM
    super-time-stepping for unsteady flows).

Every function here is pinned by the `-m "not gpu"` tests in
`tests/test_oracle_*.py` (conservation, fixed point, Poiseuille, Taylor-Green,
bounce-back permutation, brute-force DFT, library FFT, parameter counts).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

from . import fno_oracle  # noqa: F401  (re-exported)
from .fno_oracle import fno_forward, param_count  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

BC_PERIODIC, BC_PRESSURE, BC_VELOCITY = 0, 1, 2
Q = 9


_LIB_OMP = os.path.join(_HERE, "liblbm_oracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the C oracle if it is missing or stale: plain -O2, single thread (the parity
    reference), or with -fopenmp, where the row loops of collision and streaming run on
    all host cores (every cell is independent, so the results are identical)."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c99", *flags, "-shared", "-fPIC", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class _OlGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_double),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("bc_west", ctypes.c_int), ("bc_east", ctypes.c_int),
                ("west_value", ctypes.c_double), ("east_value", ctypes.c_double)]


@dataclasses.dataclass
class Grid:
    """One lattice: size, relaxation time, body force and x-end boundary kinds."""
    nx: int
    ny: int
    tau: float
    fx: float = 0.0
    fy: float = 0.0
    bc_west: int = BC_PERIODIC
    bc_east: int = BC_PERIODIC
    west_value: float = 1.0
    east_value: float = 1.0

    def c(self) -> _OlGrid:
        return _OlGrid(self.nx, self.ny, self.tau, self.fx, self.fy, self.bc_west,
                       self.bc_east, self.west_value, self.east_value)


_lib: Optional[ctypes.CDLL] = None
_lib_omp: Optional[ctypes.CDLL] = None


def lib(openmp: bool = False) -> ctypes.CDLL:
    """The single-thread oracle library, or its OpenMP build."""
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            _lib_omp = _declare(ctypes.CDLL(build(openmp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L: ctypes.CDLL) -> ctypes.CDLL:
    P = ctypes.POINTER
    d, u8 = P(ctypes.c_double), P(ctypes.c_uint8)
    g = P(_OlGrid)
    for name, args in [
        ("ol_equilibrium", [ctypes.c_double, ctypes.c_double, ctypes.c_double, d]),
        ("ol_collide", [g, u8, d, d]),
        ("ol_stream", [g, u8, d, d]),
        ("ol_boundary", [g, u8, d]),
        ("ol_run", [g, u8, d, ctypes.c_int]),
        ("ol_macro", [g, u8, d, d, d, d]),
        ("ol_reinit", [g, u8, d, d, d, ctypes.c_int, d]),
        ("ol_lattice", [P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), d]),
    ]:
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = None
    return L


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _mask(solid: np.ndarray, grid: Grid) -> np.ndarray:
    m = np.ascontiguousarray(solid, dtype=np.uint8)
    assert m.shape == (grid.ny, grid.nx)
    return m


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def lattice():
    """(cx, cy, w, opp) of the D2Q9 lattice as the C oracle defines it."""
    cx = (ctypes.c_int * Q)()
    cy = (ctypes.c_int * Q)()
    opp = (ctypes.c_int * Q)()
    w = (ctypes.c_double * Q)()
    lib().ol_lattice(cx, cy, opp, w)
    return (np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(opp[:]))


def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(Q)
    lib().ol_equilibrium(rho, ux, uy, _dp(out))
    return out


def collide(grid: Grid, solid: np.ndarray, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    m = _mask(solid, grid)
    gc = grid.c()
    lib().ol_collide(ctypes.byref(gc), _u8(m), _dp(f), _dp(out))
    return out


def stream(grid: Grid, solid: np.ndarray, fstar: np.ndarray) -> np.ndarray:
    """Streaming with halfway bounce-back, then Zou-He completion."""
    fstar = np.ascontiguousarray(fstar, dtype=np.float64)
    out = np.empty_like(fstar)
    m = _mask(solid, grid)
    gc = grid.c()
    lib().ol_stream(ctypes.byref(gc), _u8(m), _dp(fstar), _dp(out))
    return out


def boundary(grid: Grid, solid: np.ndarray, f: np.ndarray) -> np.ndarray:
    f = np.array(f, dtype=np.float64, order="C")
    m = _mask(solid, grid)
    gc = grid.c()
    lib().ol_boundary(ctypes.byref(gc), _u8(m), _dp(f))
    return f


def run(grid: Grid, solid: np.ndarray, f: np.ndarray, nsteps: int,
        openmp: bool = False) -> np.ndarray:
    """nsteps of collide + stream; returns the post-stream populations."""
    f = np.array(f, dtype=np.float64, order="C")
    m = _mask(solid, grid)
    gc = grid.c()
    lib(openmp).ol_run(ctypes.byref(gc), _u8(m), _dp(f), int(nsteps))
    return f


def macro(grid: Grid, solid: np.ndarray, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.empty((grid.ny, grid.nx))
    ux = np.empty_like(rho)
    uy = np.empty_like(rho)
    m = _mask(solid, grid)
    gc = grid.c()
    lib().ol_macro(ctypes.byref(gc), _u8(m), _dp(f), _dp(rho), _dp(ux), _dp(uy))
    return rho, ux, uy


def reinit(grid: Grid, solid: np.ndarray, rho, ux, uy, neq_mode: int = 1) -> np.ndarray:
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ux = np.ascontiguousarray(ux, dtype=np.float64)
    uy = np.ascontiguousarray(uy, dtype=np.float64)
    f = np.empty((Q, grid.ny, grid.nx))
    m = _mask(solid, grid)
    gc = grid.c()
    lib().ol_reinit(ctypes.byref(gc), _u8(m), _dp(rho), _dp(ux), _dp(uy), int(neq_mode), _dp(f))
    return f


def rest_state(grid: Grid, solid: np.ndarray) -> np.ndarray:
    """Default initialisation of Fig. 1: rho = 1, u = 0, f = f^eq (Zou-He completed)."""
    one = np.ones((grid.ny, grid.nx))
    zero = np.zeros_like(one)
    return reinit(grid, solid, one, zero, zero, neq_mode=0)


def derivative(grid: Grid, solid: np.ndarray, v, axis: int) -> np.ndarray:
    """d v / d x (axis 0) or d v / d y (axis 1) at every fluid cell: central where both
    neighbours along the axis are fluid cells of the domain, one-sided where only one
    is, zero where none is (y periodic; x periodic only for periodic grids).  The
    velocity-gradient estimate of the re-initialisation and of the vorticity."""
    v = np.asarray(v, dtype=np.float64)
    fluid = ~np.asarray(solid, dtype=bool)
    ax = 1 if axis == 0 else 0
    vp, vm = np.roll(v, -1, axis=ax), np.roll(v, 1, axis=ax)
    fp, fm = np.roll(fluid, -1, axis=ax), np.roll(fluid, 1, axis=ax)
    if axis == 0 and grid.bc_west != BC_PERIODIC:
        fp[:, -1] = False
        fm[:, 0] = False
    d = np.where(fp & fm, 0.5 * (vp - vm), np.where(fp, vp - v, np.where(fm, v - vm, 0.0)))
    return np.where(fluid, d, 0.0)


def vorticity(grid: Grid, solid: np.ndarray, ux, uy) -> np.ndarray:
    """omega = d u_y / d x - d u_x / d y (the vorticity of the unsteady error metric,
    Sec. 3.2.2); 0 at solid cells."""
    return derivative(grid, solid, uy, 0) - derivative(grid, solid, ux, 1)


def steady_residual(solid: np.ndarray, ux_now, uy_now, ux_prev, uy_prev) -> float:
    """r = ||u^n - u^(n-K)||_2 / ||u^n||_2 over fluid cells (steady-state criterion)."""
    fl = ~np.asarray(solid, dtype=bool)
    num = np.sum((ux_now - ux_prev)[fl] ** 2 + (uy_now - uy_prev)[fl] ** 2)
    den = np.sum(ux_now[fl] ** 2 + uy_now[fl] ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float("inf")


def clamp_macro(rho, ux, uy, rho_lo=0.9, rho_hi=1.1, u_max=0.2):
    """Clamp predicted fields before re-initialisation: rho into [rho_lo, rho_hi], |u| <= u_max."""
    rho = np.clip(rho, rho_lo, rho_hi)
    sp = np.sqrt(ux * ux + uy * uy)
    scale = np.where(sp > u_max, u_max / np.maximum(sp, 1e-300), 1.0)
    return rho, ux * scale, uy * scale


def fno_input(solid: np.ndarray, rho, ux, uy) -> np.ndarray:
    """FNO input channels (rho - 1, u_x, u_y, mask) as [4, ny, nx] float64."""
    return np.stack([rho - 1.0, ux, uy, np.asarray(solid, dtype=np.float64)])


ALL_CHANNELS = (0, 1, 2, 3)  # indices into the input planes (rho - 1, u_x, u_y, mask)


def fno_predict(solid, rho, ux, uy, nets, activation="gelu", clamp=(0.9, 1.1, 0.2)):
    """One FNO step on the macroscopic fields (Sec. 2.3), clamped.

    nets: ((shape, params, channels),) for one network mapping the selected input planes
    to (delta rho, u_x, u_y), or ((shape_rho, params_rho, channels_rho), (shape_u,
    params_u, channels_u)) for a density network (one output, delta rho) and a velocity
    network (two outputs, u_x and u_y), as the paper's model groups are built.  Both
    networks read the fields of the same time level."""
    planes = fno_input(solid, rho, ux, uy)
    outs = [fno_forward(sh, pa, planes[list(ch)][None], activation=activation)[0]
            for sh, pa, ch in nets]
    if len(nets) == 1:
        dr, vx, vy = outs[0]
    else:
        dr, (vx, vy) = outs[0][0], outs[1]
    return clamp_macro(1.0 + dr, vx, vy, *clamp)


def hybrid_steady(grid: Grid, solid: np.ndarray, shape, params, nsteps: int,
                  check_every: int = 100, neq_mode: int = 1, use_fno: bool = True,
                  activation: str = "gelu", clamp=(0.9, 1.1, 0.2), nets=None):
    """Steady framework (Fig. 3a): FNO prediction -> re-initialisation -> LBM.

    The FNO sees the default fields (rho = 1, u = 0) and the mask; its output
    (delta rho, u_x, u_y) is clamped and turned into populations.  `nets` overrides the
    single (shape, params) network (see fno_predict).  Returns (f, residual history
    [(step, r)]).

    The residual at a check compares u with the velocity of the previous check; before
    the first check that is the velocity the start prescribed (zero from rest, the
    clamped prediction from the FNO), so the first residual from rest is 1.
    """
    one = np.ones((grid.ny, grid.nx))
    zero = np.zeros_like(one)
    if use_fno:
        nets = nets or ((shape, params, ALL_CHANNELS),)
        rho, ux, uy = fno_predict(solid, one, zero, zero, nets, activation, clamp)
        f = reinit(grid, solid, rho, ux, uy, neq_mode)
        fl = ~np.asarray(solid, dtype=bool)
        ux_p, uy_p = np.where(fl, ux, 0.0), np.where(fl, uy, 0.0)
    else:
        f = rest_state(grid, solid)
        ux_p, uy_p = zero, zero
    hist = []
    done = 0
    while done < nsteps:
        k = min(check_every, nsteps - done)
        f = run(grid, solid, f, k)
        done += k
        _, ux_n, uy_n = macro(grid, solid, f)
        hist.append((done, steady_residual(solid, ux_n, uy_n, ux_p, uy_p)))
        ux_p, uy_p = ux_n, uy_n
    return f, hist


def hybrid_unsteady(grid: Grid, solid: np.ndarray, shape, params, f0: np.ndarray,
                    k_lbm: int, m_fno: int, cycles: int, neq_mode: int = 1,
                    activation: str = "gelu", clamp=(0.9, 1.1, 0.2), nets=None):
    """Super-time-stepping (Fig. 3b): per cycle k_lbm LBM steps, then m_fno FNO
    steps on the macroscopic fields, then re-initialisation of f.  `nets` overrides
    the single (shape, params) network (see fno_predict).  Returns f."""
    nets = nets or ((shape, params, ALL_CHANNELS),)
    f = np.array(f0, dtype=np.float64)
    for _ in range(cycles):
        f = run(grid, solid, f, k_lbm)
        rho, ux, uy = macro(grid, solid, f)
        for _ in range(m_fno):
            rho, ux, uy = fno_predict(solid, rho, ux, uy, nets, activation, clamp)
        f = reinit(grid, solid, rho, ux, uy, neq_mode)
    return f
