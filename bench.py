#!/usr/bin/env python3
"""Benchmark of the hybrid FNO-LBM hot path on GB300.

Workload (per GPU): porous-media steady state, a batch of T trajectories of
512 x 256 lattices (pressure inlet rho = 1.001, outlet rho = 1.0, periodic sides,
tau = 0.7, non-overlapping seeded disks of radius 4-12 at porosity U(0.6, 0.8)).
One *step* is one full pass of the hot path over the batch:
  FNO prediction (4 layers, 32 channels, 12 x 12 modes, BF16) on (rho-1, u, mask)
  -> clamp -> re-initialisation f = f^eq + f^neq -> fused D2Q9 BGK steps with the
  residual ||u^n - u^(n-100)|| / ||u^n|| checked every 100 steps (FP64
  reductions) until it is below 1e-7 for every trajectory or a cap of
  --solve-steps LBM steps (this porous medium relaxes diffusively, so a full
  solve to 1e-7 takes far longer than a benchmark step).
metric: GLUPS = lattice-cell updates (all cells) per second over the timed steps.
Extra fields: roofline of the step kernel (CUDA events, committed ncu traffic record);
time to steady state of the FNO-initialised and of the plain (rest-state) start at the
same tolerance (steady driver), and a tolerance ladder 1e-3 ... 1e-7 over rest,
random-weight-FNO and trained-FNO starts (the FNO trained here on LBM steady states of
other geometries); large single-domain sweep; FNO throughput; batched unsteady
super-time-stepping; double shear layer at 1:1 / 1:2 / 1:3; the differentiable training
step; the CPU oracle timed on the host; clocks; e2e through the Python/C API.

Multi-GPU (torchrun): trajectories are independent; every rank solves its own
batch (seeds offset by rank), no data-path collective -> weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D2Q9 GLUPS (% HBM peak); time-to-steady hybrid vs plain LBM, same tol"
NX, NY = 512, 256
TAU, RHO_IN, RHO_OUT = 0.7, 1.001, 1.0
TOL, CHECK_EVERY = 1e-7, 100
BYTES_PER_CELL = 72.125  # 9 x 4 B read + 9 x 4 B written + 1 mask bit per cell update
REINIT_BYTES_PER_CELL = 56  # (rho, u_x, u_y) read; 9 populations + stored (u_x, u_y) written


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--trajectories", type=int, default=64)
    ap.add_argument("--solve-steps", type=int, default=20000,
                    help="LBM step cap of the solve inside one benchmark step")
    ap.add_argument("--tts-trajectories", type=int, default=20)
    ap.add_argument("--tts-max-steps", type=int, default=150000)
    ap.add_argument("--tts-tol", type=float, default=1e-5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--unsteady-trajectories", type=int, default=100)
    ap.add_argument("--unsteady-cycles", type=int, default=20)
    ap.add_argument("--ladder-trajectories", type=int, default=20,
                    help="trajectories of the tolerance ladder (steps to 1e-4 ... 1e-7, both starts)")
    ap.add_argument("--ladder-max-steps", type=int, default=100000)
    ap.add_argument("--train-samples", type=int, default=128,
                    help="LBM steady states used to train the initialisation FNO (0: no trained arm)")
    ap.add_argument("--train-lbm-steps", type=int, default=50000)
    ap.add_argument("--train-fno-steps", type=int, default=1500)
    ap.add_argument("--no-sweep", action="store_true", help="skip the large-domain LBM sweep")
    ap.add_argument("--shear-trajectories", type=int, default=100,
                    help="double-shear-layer trajectories (0: skip the workload)")
    ap.add_argument("--train-steps", type=int, default=5,
                    help="timed steps of the differentiable hybrid training workload (0: skip)")
    ap.add_argument("--step-variant", type=int, default=-1,
                    help="step-kernel tile shape index; -1 (default) times all shapes and keeps the fastest")
    ap.add_argument("--case", default=None,
                    choices=["lbm", "check", "reinit", "fno", "shear_fno"],
                    help="run one small case to be profiled and exit (no JSON line): 'lbm' 60 "
                         "steps of the bench batch (tile shape 3), 'check' 5 steps + 5 "
                         "statistics-only residuals + 5 step+statistics checks of it, "
                         "'reinit' 5 re-initialisations of it from its fields after 20 steps, 'fno' "
                         "8 forwards of the FNO throughput shape, 'shear_fno' 8 forwards of "
                         "the double-shear density and velocity networks on 100 fields")
    return ap.parse_args()


def run_case(args):
    """Small cases for ncu captures (one kernel, few launches before the captured ones)."""
    import torch
    import synth
    import paper_2604_27158_gb300 as P
    from paper_2604_27158_gb300.fno import Fno, FnoShape
    from paper_2604_27158_gb300.lbm import GridSpec, Lattice
    if args.case in ("lbm", "check"):
        T = args.trajectories
        masks, _ = workload(T, 0)
        lat = Lattice([GridSpec(NX, NY, TAU, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                                west_value=RHO_IN, east_value=RHO_OUT)] * T, masks)
        lat.set_step_variant(3 if args.step_variant < 0 else args.step_variant)
        if args.case == "lbm":
            lat.step(60)
        else:
            lat.step(20)
            for _ in range(5):
                lat.step(1)
            for _ in range(5):
                lat.residual(update_prev=True)
            for _ in range(5):
                lat.step_residual(update_prev=True)
        lat.close()
    elif args.case == "reinit":
        T = args.trajectories
        masks, _ = workload(T, 0)
        lat = Lattice([GridSpec(NX, NY, TAU, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                                west_value=RHO_IN, east_value=RHO_OUT)] * T, masks)
        lat.step(20)
        rho, ux, uy = lat.macro()
        for _ in range(5):
            lat.reinit(rho, ux, uy, neq_mode=1)
        lat.close()
    elif args.case == "shear_fno":
        ics = synth.double_shear(100, seed=2000)
        n = ics[0]["rho"].shape[0]
        xr = torch.from_numpy(np.stack([ic["rho"] - 1.0 for ic in ics])[:, None].astype(np.float32)).cuda()
        xu = torch.from_numpy(np.stack([np.stack([ic["ux"], ic["uy"]]) for ic in ics]).astype(np.float32)).cuda()
        nets = []
        for cin, modes, seed, x in ((1, 8, 31, xr), (2, 32, 32, xu)):
            sh = synth.FnoShape(c_in=cin, c_out=cin, width=14, layers=3, modes=modes,
                                dec_size=32, padding=9)
            nets.append((Fno(FnoShape(c_in=cin, c_out=cin, width=14, layers=3, modes=modes,
                                      dec_size=32, padding=9),
                             synth.fno_flatten_params(sh, synth.fno_random_params(sh, seed=seed))),
                         x, torch.empty_like(x)))
        for _ in range(8):
            for net, x, y in nets:
                net(x, y)
        for net, _, _ in nets:
            net.check(100, n, n)
            net.close()
    else:
        B = 32
        sshape, flat = fno_params()
        net = Fno(FnoShape(), flat)
        x = torch.randn(B, 4, 256, 256, device="cuda") * 1e-2
        y = torch.empty(B, 3, 256, 256, device="cuda")
        for _ in range(8):
            net(x, y)
        net.check(B, 256, 256)
        net.close()
    torch.cuda.synchronize()
    return 0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed0(rank, T):
    """First geometry seed of a rank: ranks draw disjoint seed ranges (independent batches)."""
    return rank * T


def reduce_over_ranks(ms, updates, world, device):
    """Job time = slowest rank; work = sum over ranks.  The only collectives of the run."""
    if world <= 1:
        return ms, updates
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], device=device, dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def step_kernel_traffic(cells, shape):
    """DRAM bytes per step-kernel launch from the committed ncu record of the tile shape in
    use, scaled to `cells`; None when there is no record for that shape or the step kernel's
    source changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k_step_tma_traffic.json")))
        src = open(os.path.join(ROOT, "paper_2604_27158_gb300", "csrc", "lbm.cu")).read()
        a = src.index("// ------------------------------------------------------ the fused step ---")
        b = src.index("__global__ void __launch_bounds__(kBlock) k_export(")
        if hashlib.sha256(src[a:b].encode()).hexdigest()[:16] != rec["source_section_sha256_16"]:
            return None
        if rec["variant"] != shape[0]:
            return None
        return rec["traffic_bytes_per_launch"] * cells / rec["cells"]
    except Exception:
        return None


def fno_flops(B, H, W, C=32, m=12, layers=4, cin=4, S=32, cout=3):
    """Algorithmic FLOPs of one FNO forward (separable truncated DFTs, Sec. 2.2 layer equation)."""
    px = B * H * W
    layer = (2 * 2 * m * W * B * H * C          # forward x-DFT over the kept kx
             + 8 * 2 * m * H * m * B * C        # forward y-DFT over the kept ky (complex)
             + 8 * C * C * 2 * m * m * B        # per-mode complex channel mixing
             + 8 * 2 * m * H * m * B * C        # inverse y-DFT
             + 2 * 2 * m * W * B * H * C        # inverse x-DFT (real output)
             + 2 * C * C * px)                  # 1x1 convolution W
    lift = 2 * ((cin + 2) * C // 2 + C // 2 * C) * px
    dec = 2 * (C * S + S * cout) * px
    return layers * layer + lift + dec


def fno_bytes(B, H, W, C=32, layers=4, cin=4, cout=3):
    """Algorithmic HBM bytes of one FNO forward with fused layer boundaries: every layer
    reads and writes its BF16 latent field once; FP32 input and output fields."""
    return layers * 2 * B * H * W * C * 2 + B * H * W * (cin + cout) * 4


def fno_snapshot_inputs(P, GridSpec, Lattice, B, H, W, steps=2000):
    """FNO inputs (rho-1, ux, uy, mask) from LBM snapshots: B body-force channels of H x W
    with walls and 6 seeded disks (radius 4-8 scaled by W/128), tau 0.8, after `steps` steps."""
    import synth
    import torch
    masks = [synth.channel_with_disks(W, H, 6, 4 * W // 128, 8 * W // 128, seed=b)[0]
             for b in range(B)]
    lat = Lattice([GridSpec(W, H, 0.8, fx=1e-6) for _ in range(B)], masks)
    lat.step(steps)
    rho, ux, uy = lat.macro()
    m = torch.from_numpy(np.stack(masks).astype(np.float32)).cuda()
    x = torch.stack([rho.view(B, H, W) - 1.0, ux.view(B, H, W), uy.view(B, H, W), m], dim=1)
    torch.cuda.synchronize()
    lat.close()
    return x.contiguous()


def tiled_porous(nx, ny, seed, ntiles=8, porosity=0.7):
    """A large porous domain built from seeded 512 x 256 tiles of the porous-media generator
    at a fixed porosity (the tiles keep their disks away from the tile's x edges)."""
    import synth
    tiles = [synth.porous_media(NX, NY, 4, 12, porosity_range=(porosity, porosity), seed=seed + k)[0]
             for k in range(ntiles)]
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, ntiles, size=(ny // NY, nx // NX))
    return np.block([[tiles[k] for k in row] for row in pick])


def workload(T, seed0):
    import synth
    masks, phis = [], []
    for k in range(T):
        solid, _, phi = synth.porous_media(NX, NY, 4, 12, seed=seed0 + k)
        masks.append(solid)
        phis.append(phi)
    return masks, phis


def fno_params(seed=0):
    import synth
    shape = synth.FnoShape(c_in=4, c_out=3, width=32, layers=4, modes=12, dec_layers=1, dec_size=32)
    return shape, synth.fno_flatten_params(shape, synth.fno_random_params(shape, seed=seed))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 6:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[2:6]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_glups(g, solid, budget_s, openmp):
    import oracle
    f = oracle.rest_state(g, solid)
    t0 = time.perf_counter()
    f = oracle.run(g, solid, f, 10, openmp=openmp)
    dt = time.perf_counter() - t0
    n = max(10, int(budget_s / max(dt / 10, 1e-9)))
    t0 = time.perf_counter()
    oracle.run(g, solid, f, n, openmp=openmp)
    dt = time.perf_counter() - t0
    return NX * NY * n / dt / 1e9, n, dt


def cpu_baseline(masks, budget_s=8.0):
    """The FP64 C oracle on one trajectory, bounded to ~budget_s per build: the OpenMP build
    on all host cores (the reported value) and the single-thread parity build."""
    import oracle
    g = oracle.Grid(nx=NX, ny=NY, tau=TAU, bc_west=oracle.BC_PRESSURE, bc_east=oracle.BC_PRESSURE,
                    west_value=RHO_IN, east_value=RHO_OUT)
    cores = os.cpu_count() or 1
    v1, n1, dt1 = _oracle_glups(g, masks[0], budget_s, openmp=False)
    try:
        vm, nm, dtm = _oracle_glups(g, masks[0], budget_s, openmp=True)
    except Exception as e:  # no OpenMP runtime: report the single-thread build only
        return {"value": v1, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                "sample": f"FP64 C oracle, 1 thread ({type(e).__name__} building the OpenMP "
                          f"oracle): {n1} LBM steps of one 512x256 porous trajectory in {dt1:.1f} s"}
    return {"value": vm, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle, OpenMP rows on {cores} host threads: {nm} LBM steps of one "
                      f"512x256 porous trajectory (seed 0) in {dtm:.1f} s",
            "single_thread": {"value": v1, "unit": "GLUPS", "cores": 1,
                              "sample": f"{n1} steps in {dt1:.1f} s"},
            "fno_oracle": fno_oracle_baseline()}


def fno_oracle_baseline(reps=2):
    """The FP64 numpy FNO oracle (naive truncated DFTs as BLAS matrix products) on the
    FNO throughput workload's shape, timed at B = 1 and scaled x32."""
    import oracle
    import synth
    shape, _ = fno_params()
    params = synth.fno_random_params(shape, seed=0)
    x = np.random.default_rng(0).standard_normal((1, 4, 256, 256)) * 1e-2
    oracle.fno_forward(shape, params, x)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.fno_forward(shape, params, x)
    ms1 = 1e3 * (time.perf_counter() - t0) / reps
    return {"ms_per_forward_b32": 32 * ms1, "ms_per_forward_b1": ms1,
            "sample": f"B=1 x 256 x 256 forward (4 layers, 32 channels, 12x12 modes), {reps} "
                      f"runs, scaled x32; numpy BLAS threads on the host"}


def bench_config(T, phis, solve_steps, world):
    cells = T * NX * NY
    return {"workload": f"porous-media steady state, {T} trajectories of {NX}x{NY} per GPU "
                        f"(tau {TAU}, rho_in {RHO_IN}, rho_out {RHO_OUT}, disks r 4-12, "
                        f"porosity {min(phis):.3f}-{max(phis):.3f}); step = FNO init "
                        f"(4x32ch, 12x12 modes, BF16) + reinit + LBM until residual < {TOL:g} "
                        f"or {solve_steps} steps",
            "trajectories_per_gpu": T, "cells_per_gpu": cells,
            "lbm_steps_per_step": solve_steps, "l2": "working set "
            f"{2 * 36 * cells / 1e6:.0f} MB of populations per step > 129 MB L2, no flush",
            "parallelism": f"independent trajectories x{world}"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    masks, phis = workload(args.trajectories, 0)
    samples = []
    for _ in range(args.warmup):
        cpu_baseline(masks, budget_s=1.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        samples.append(cpu_baseline(masks, budget_s=6.0))
    wall = time.perf_counter() - t0
    v = float(np.mean([s["value"] for s in samples]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args.trajectories, phis, args.solve_steps, 1),
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": samples[0]["cores"],
                             "kind": "oracle",
                             "sample": "each step: " + samples[0]["sample"] + " (a bounded sample "
                                       "of the workload; GLUPS is per cell update, as in ours)"},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case is not None:
        return run_case(args)
    rank, world, local = dist_env()
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2604_27158_gb300 as P
    from paper_2604_27158_gb300.fno import Fno, FnoShape, Hybrid, HybridConfig
    from paper_2604_27158_gb300.lbm import GridSpec, Lattice

    T = args.trajectories
    masks, phis = workload(T, seed0=rank_seed0(rank, T))
    grids = [GridSpec(NX, NY, TAU, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                      west_value=RHO_IN, east_value=RHO_OUT) for _ in range(T)]
    sshape, flat = fno_params()
    net = Fno(FnoShape(), flat)
    lat = Lattice(grids, masks)
    cells = lat.cells
    if args.step_variant >= 0:
        lat.set_step_variant(args.step_variant)
        tune_ms = None
    else:
        _, tune_ms = lat.autotune(reps=20)
    shape = lat.step_variant()
    hyb = Hybrid(lat, net, HybridConfig(use_fno=1, neq_mode=1, check_every=CHECK_EVERY, tol=TOL,
                                        max_steps=args.solve_steps))
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        hyb.advance()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_updates = 0
    info = None
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            st, first, res = hyb.advance()
            total_updates += int(st.steps) * cells
            info = (st, first, res)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    t_max, total_updates = reduce_over_ranks(ms, total_updates, world, "cuda")
    glups = total_updates / (t_max * 1e-3) / 1e9
    st, first, res = info

    # dominant kernel: the fused step, timed alone with CUDA events on the launching stream
    lat.step(20)
    nk = 400
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    lat.step(nk)
    k1.record(stream)
    torch.cuda.synchronize()
    kms = k0.elapsed_time(k1) / nk
    peak, peak_kind = read_peaks()
    achieved = BYTES_PER_CELL * cells / (kms * 1e-3) / 1e9

    # the re-initialisation kernel (a4) on the same batch, from its macroscopic fields: reads
    # (rho, u_x, u_y), writes the nine populations and the stored velocity (56 B a cell;
    # 470 MB a launch at this size, well above the L2)
    rho_m, ux_m, uy_m = lat.macro()
    for _ in range(3):
        lat.reinit(rho_m, ux_m, uy_m, neq_mode=1)
    nr = 20
    k0.record(stream)
    for _ in range(nr):
        lat.reinit(rho_m, ux_m, uy_m, neq_mode=1)
    k1.record(stream)
    torch.cuda.synchronize()
    rms = k0.elapsed_time(k1) / nr
    reinit_gbs = REINIT_BYTES_PER_CELL * cells / (rms * 1e-3) / 1e9
    reinit_kernel = {"kernel": "k_reinit", "neq_mode": 1, "launch_ms": rms,
                     "bytes_per_launch": REINIT_BYTES_PER_CELL * cells, "achieved_gbs": reinit_gbs,
                     "frac_of_measured_hbm": reinit_gbs / peak}
    del rho_m, ux_m, uy_m

    tts = None

    # tolerance ladder (Table 1 of the paper reports outputs to 1e-4 ... 2e-7): per trajectory,
    # the first check step at which r < eps, on a batch of --ladder-trajectories
    # trajectories with a step cap; geometric mean over trajectories.  Three starts: rest
    # state, the seeded random-weight FNO, and an FNO trained here on LBM steady states
    # of other geometries of the same generator (the paper's offline training, Sec. 2.3).
    ladder = None
    if args.ladder_trajectories > 0:
        from paper_2604_27158_gb300 import steady_training as stt
        import synth
        Tl = min(args.ladder_trajectories, T)
        eps_list = [1e-3, 1e-4, 1e-5, 1e-6, 2e-7, 1e-7]
        trained = None
        if args.train_samples > 0:
            tr0 = time.perf_counter()
            tmasks_tr = [synth.porous_media(NX, NY, 4, 12, seed=50000 + k)[0]
                         for k in range(args.train_samples)]
            y_tr = stt.steady_states(grids[0], tmasks_tr, args.train_lbm_steps)
            x_tr = stt.fno_inputs(tmasks_tr)
            fl_tr = ~torch.from_numpy(np.stack(tmasks_tr)).cuda()
            tparams, thist = stt.train_supervised(FnoShape(), synth.fno_flatten_params(
                sshape, synth.fno_random_params(sshape, seed=7, out_scale=1.0)), x_tr, y_tr,
                fl_tr, args.train_fno_steps, batch=8, lr=2e-3, seed=0, log_every=100)
            torch.cuda.synchronize()
            trained = Fno(FnoShape(), tparams)
            # prediction error on the ladder's (held-out) geometries against their states
            # after the same number of LBM steps
            y_ev = stt.steady_states(grids[0], masks[:Tl], args.train_lbm_steps)
            pred = torch.empty_like(y_ev)
            trained(stt.fno_inputs(masks[:Tl]), pred)
            fl_ev = ~torch.from_numpy(np.stack(masks[:Tl])).cuda()
            pred_err = [float((pred[:, c] - y_ev[:, c])[fl_ev].norm() / y_ev[:, c][fl_ev].norm())
                        for c in range(3)]
            trained_info = {"samples": args.train_samples, "lbm_steps_per_sample": args.train_lbm_steps,
                            "optimiser_steps": args.train_fno_steps, "batch": 8,
                            "seconds": time.perf_counter() - tr0,
                            "loss_every_100": thist,
                            "heldout_rel_l2_rho_ux_uy": pred_err}
            del x_tr, y_tr, y_ev, pred
        lat_l = Lattice(grids[:Tl], masks[:Tl])
        lat_l.set_step_variant(shape[0])
        arms = {}
        finals = {}
        arm_list = [("plain_init", None), ("fno_random_init", net)]
        if trained is not None:
            arm_list.append(("fno_trained_init", trained))
        for name, anet in arm_list:
            h_l = Hybrid(lat_l, anet, HybridConfig(use_fno=1 if anet is not None else 0,
                                                   neq_mode=1, check_every=CHECK_EVERY,
                                                   tol=1e-30, max_steps=CHECK_EVERY))
            first = np.full((len(eps_list), Tl), -1, dtype=np.int64)
            t_all = [None] * len(eps_list)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            _, _, r = h_l.advance()  # init (+ FNO and reinit) and the first CHECK_EVERY steps
            n = CHECK_EVERY
            while True:
                for e, eps in enumerate(eps_list):
                    hit = (first[e] < 0) & (r < eps)
                    first[e][hit] = n
                    if t_all[e] is None and (first[e] >= 0).all():
                        t_all[e] = time.perf_counter() - w0
                if (first[-1] >= 0).all() or n >= args.ladder_max_steps:
                    break
                lat_l.step(CHECK_EVERY)
                n += CHECK_EVERY
                r = lat_l.residual(update_prev=True, raise_unstable=False)[:, 0]
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
            h_l.close()
            rows = {}
            for e, eps in enumerate(eps_list):
                ok = first[e] > 0
                rows[f"{eps:g}"] = {
                    "reached": int(ok.sum()),
                    "geomean_steps": float(np.exp(np.mean(np.log(first[e][ok])))) if ok.any() else None,
                    "seconds_until_all_reached": t_all[e],
                    "steps": [int(v) for v in first[e]]}
            arms[name] = {"per_tol": rows, "steps_run": n, "seconds": wall}
            _, fux, fuy = lat_l.macro()
            finals[name] = torch.stack([fux, fuy])
        # equal final accuracy: the starts approach the same steady state
        for name in list(arms):
            if name != "plain_init":
                dq = (finals[name] - finals["plain_init"]).norm() / finals["plain_init"].norm()
                arms[name]["final_u_rel_diff_vs_plain"] = float(dq)
        lat_l.close()
        ladder = {"trajectories": Tl, "step_cap": args.ladder_max_steps, "check_every": CHECK_EVERY,
                  "residual": "||u^n - u^(n-100)|| / ||u^n|| over fluid cells (FP64 on the GPU)",
                  **arms,
                  "trained_fno": trained_info if trained is not None else None,
                  "note": "steps to tol exclude nothing: the FNO start includes the FNO forward "
                          "and the reinit in its wall time; host synchronisation every 100 steps "
                          "applies to every arm alike"}
        # time to steady through the library's steady driver (hybrid_advance): plain start
        # vs the trained-FNO start, same tolerance, same trajectories
        if args.tts_trajectories > 0:
            Tt = min(args.tts_trajectories, Tl)
            lat_t = Lattice(grids[:Tt], masks[:Tt])
            lat_t.set_step_variant(shape[0])
            tarms = {}
            tnet = trained if trained is not None else net
            for name, anet in (("fno_init", tnet), ("plain_init", None)):
                h_t = Hybrid(lat_t, anet, HybridConfig(use_fno=1 if anet is not None else 0,
                                                       neq_mode=1, check_every=CHECK_EVERY,
                                                       tol=args.tts_tol,
                                                       max_steps=args.tts_max_steps))
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                ast, afirst, ares = h_t.advance()
                a1.record(stream)
                torch.cuda.synchronize()
                tarms[name] = {"seconds": a0.elapsed_time(a1) / 1e3, "steps": int(ast.steps),
                               "converged": bool(ast.converged),
                               "steps_to_tol": [int(v) for v in afirst],
                               "final_residual": [float(v) for v in ares]}
                h_t.close()
            lat_t.close()
            tts = {"tol": args.tts_tol, "check_every": CHECK_EVERY, "trajectories": Tt,
                   "step_cap": args.tts_max_steps, "driver": "hybrid_advance (steady mode)",
                   "fno_init": tarms["fno_init"], "plain_init": tarms["plain_init"],
                   "speedup_wall": (tarms["plain_init"]["seconds"] / tarms["fno_init"]["seconds"]
                                    if tarms["fno_init"]["converged"] else None),
                   "fno": ("FNO trained here on LBM steady states of other geometries"
                           if trained is not None else "seeded random weights")}
        if trained is not None:
            trained.close()

    # large single domains of the same porous generator at porosity 0.7 (1 GPU, rank 0):
    # the step kernel alone, 200 warm-up steps then 1000 timed steps
    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = []
        for (sx, sy) in ((4096, 4096), (8192, 8192), (16384, 8192)):
            solid = tiled_porous(sx, sy, seed=77)
            gs = GridSpec(sx, sy, TAU, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                          west_value=RHO_IN, east_value=RHO_OUT)
            lat_s = Lattice([gs], [solid])
            _, sw_ms = lat_s.autotune(reps=5)
            sv = lat_s.step_variant()
            lat_s.step(200)
            w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            w0.record(stream)
            lat_s.step(1000)
            w1.record(stream)
            torch.cuda.synchronize()
            sms = w0.elapsed_time(w1) / 1000
            cells_s = sx * sy
            fluid_s = int((~solid).sum())
            gl = cells_s / (sms * 1e-3) / 1e9
            sweep.append({"nx": sx, "ny": sy, "cells": cells_s, "porosity": fluid_s / cells_s,
                          "f_bytes": 2 * 36 * cells_s, "ms_per_step": sms, "glups": gl,
                          "glups_fluid_only": fluid_s / (sms * 1e-3) / 1e9,
                          "frac_of_measured_hbm": gl * BYTES_PER_CELL / peak,
                          "frac_of_8tbs": gl * BYTES_PER_CELL / 8000.0,
                          "tile_shape": {"rows_per_tile": sv[1], "stages": sv[2],
                                         "ctas_per_sm": sv[3]}})
            lat_s.close()
            del solid

    # small, L2-resident lattices where launch cost may dominate: the 128 x 64 channel
    # (tau 0.8, g_x 1e-6, six disks r 4-8, 2000 steps) alone and as a batch of its ten
    # seeds in one launch per step, and one 512 x 256 porous trajectory; each timed with
    # one stream launch per step (programmatic dependent launch) and as CUDA graphs of
    # 100 steps
    launch_bound = None
    if rank == 0:
        import synth
        launch_bound = {}
        cases = []
        ch = [synth.channel_with_disks(128, 64, 6, 4, 8, seed=k)[0] for k in range(10)]
        gch = GridSpec(128, 64, 0.8, fx=1e-6)
        cases.append(("channel_128x64", [gch], ch[:1]))
        cases.append(("channel_128x64_x10_batch", [gch] * 10, ch))
        gpo = GridSpec(NX, NY, TAU, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                       west_value=RHO_IN, east_value=RHO_OUT)
        cases.append(("porous_512x256_one_trajectory", [gpo], masks[:1]))
        for name, gl, ml in cases:
            lat_b = Lattice(gl, ml)
            lat_b.autotune(reps=20)
            nsteps = 2000
            lat_b.step(200)
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            lat_b.step(nsteps)
            b1.record(stream)
            torch.cuda.synchronize()
            ms_stream = b0.elapsed_time(b1)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                lat_b.step(100)
            for _ in range(2):
                graph.replay()
            b0.record(stream)
            for _ in range(nsteps // 100):
                graph.replay()
            b1.record(stream)
            torch.cuda.synchronize()
            ms_graph = b0.elapsed_time(b1)
            lat_b.set_persistent(True)
            lat_b.step(200)
            b0.record(stream)
            lat_b.step(nsteps)
            b1.record(stream)
            torch.cuda.synchronize()
            ms_pers = b0.elapsed_time(b1)
            lat_b.set_persistent(False)
            cl = lat_b.cells
            sv = lat_b.step_variant()
            launch_bound[name] = {
                "cells": cl, "steps": nsteps,
                "us_per_step_stream": 1e3 * ms_stream / nsteps,
                "us_per_step_graph": 1e3 * ms_graph / nsteps,
                "glups_stream": cl * nsteps / (ms_stream * 1e-3) / 1e9,
                "glups_graph": cl * nsteps / (ms_graph * 1e-3) / 1e9,
                "us_per_step_persistent": 1e3 * ms_pers / nsteps,
                "glups_persistent": cl * nsteps / (ms_pers * 1e-3) / 1e9,
                "f_bytes": 2 * 36 * cl,
                "tile_shape": {"rows_per_tile": sv[1], "stages": sv[2], "ctas_per_sm": sv[3]}}
            del graph
            lat_b.close()
        launch_bound["note"] = ("L2-resident working sets (no HBM roofline); one launch per "
                                "step overlapped by programmatic dependent launch vs replay of "
                                "captured 100-step graphs vs all 2000 steps in one persistent "
                                "cooperative launch with a grid barrier between steps")

    # FNO throughput alone (B=32, 256x256, 4 channels -> 32 latent, 4 layers, 12x12 modes)
    fno_tp = None
    if rank == 0:
        Bf, Hf, Wf = 32, 256, 256
        xin = fno_snapshot_inputs(P, GridSpec, Lattice, Bf, Hf, Wf)
        yout = torch.empty((Bf, 3, Hf, Wf), device="cuda")
        for _ in range(3):
            net(xin, yout)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nf = 20
        f0.record(stream)
        for _ in range(nf):
            net(xin, yout)
        f1.record(stream)
        torch.cuda.synchronize()
        net.check(Bf, Hf, Wf)
        fms = f0.elapsed_time(f1) / nf
        flops = fno_flops(Bf, Hf, Wf)
        tf = flops / (fms * 1e-3) / 1e12
        try:
            pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            tpeak, tkind = float(pk["bf16_tflops"]), "measured burst"
        except Exception:
            tpeak, tkind = 1900.0, "fallback"
        try:
            tpeak_s = float(pk["bf16_tflops_sustained"])
        except Exception:
            tpeak_s = 1700.0
        fbytes = fno_bytes(Bf, Hf, Wf)
        fno_tp = {"workload": "FNO forward, batch 32 x 256 x 256, (rho-1, ux, uy, mask) snapshots "
                              "after 2000 LBM steps of 32 body-force channels with 6 disks, 32 "
                              "latent channels, 4 layers, 12x12 modes, decoder 32 -> 3, BF16 / "
                              "FP32 accumulate",
                  "ms_per_forward": fms, "gflop_per_forward": flops / 1e9, "tflops": tf,
                  "tensor_peak_tflops": tpeak, "peak_kind": tkind, "frac_of_tensor_peak": tf / tpeak,
                  "frac_of_sustained_tensor_peak": tf / tpeak_s,
                  "algorithmic_gb_per_forward": fbytes / 1e9,
                  "hbm_gbs": fbytes / (fms * 1e-3) / 1e9,
                  "frac_of_measured_hbm": fbytes / (fms * 1e-3) / 1e9 / peak,
                  "tensor_ceiling_at_this_intensity": (flops / fbytes) * peak / 1e3 / tpeak,
                  "tensor_cores": bool(net.uses_tensor_cores(Hf, Wf))}

    # batched super-time-stepping (Fig. 3b): 100 trajectories of uneven size, cycles of
    # k = 50 LBM steps + m = 5 FNO steps (Delta T = 223 Delta t each) + reinit, one CUDA
    # graph per cycle; the reference is pure LBM over the same physical time
    unsteady = None
    if rank == 0 and args.unsteady_trajectories > 0:
        import synth
        ub = synth.unsteady_batch(args.unsteady_trajectories, seed=1000)
        ug = [GridSpec(t["nx"], t["ny"], t["tau"], bc_west=P.BC_VELOCITY, bc_east=P.BC_PRESSURE,
                       west_value=t["u_in"], east_value=1.0) for t in ub]
        um = [t["solid"] for t in ub]
        lat_h = Lattice(ug, um)
        lat_r = Lattice(ug, um)
        k_lbm, m_fno, dT = 50, 5, 223
        hyb_u = Hybrid(lat_h, net, HybridConfig(mode=1, k_lbm=k_lbm, m_fno=m_fno, neq_mode=1))
        fluid = torch.from_numpy(~np.concatenate([m.ravel() for m in um])).cuda()
        # sampled trajectories (the two smallest grids) run through the FP64 oracle hybrid
        # with the same bfloat16 weights, cycle by cycle, for the per-cycle relative L2
        import oracle
        offs = np.cumsum([0] + [t["nx"] * t["ny"] for t in ub])
        sample = sorted(range(len(ub)), key=lambda i: (ub[i]["nx"] * ub[i]["ny"], i))[:2]
        o_params = synth.fno_random_params(sshape, seed=0)
        o_state = {}
        for i in sample:
            t = ub[i]
            og = oracle.Grid(nx=t["nx"], ny=t["ny"], tau=t["tau"], bc_west=oracle.BC_VELOCITY,
                             bc_east=oracle.BC_PRESSURE, west_value=t["u_in"], east_value=1.0)
            o_state[i] = (og, oracle.rest_state(og, t["solid"]))
        o_errs = {i: [] for i in sample}
        o_secs = 0.0
        cyc_ms, ref_ms, errs = [], [], []
        for c in range(args.unsteady_cycles):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            hyb_u.advance(cycles=1)
            c1.record(stream)
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            lat_r.step(k_lbm + m_fno * dT)
            r1.record(stream)
            torch.cuda.synchronize()
            cyc_ms.append(c0.elapsed_time(c1))
            ref_ms.append(r0.elapsed_time(r1))
            _, uxh, uyh = lat_h.macro()
            _, uxr, uyr = lat_r.macro()
            num = ((uxh - uxr)[fluid] ** 2 + (uyh - uyr)[fluid] ** 2).sum()
            den = (uxr[fluid] ** 2 + uyr[fluid] ** 2).sum()
            errs.append(float(torch.sqrt(num / den)))
            o0 = time.perf_counter()
            for i in sample:
                og, of = o_state[i]
                of = oracle.hybrid_unsteady(og, ub[i]["solid"], sshape, o_params, of, k_lbm,
                                            m_fno, cycles=1)
                o_state[i] = (og, of)
                _, oux, ouy = oracle.macro(og, ub[i]["solid"], of)
                fl_i = ~ub[i]["solid"]
                gx = uxh[offs[i]:offs[i + 1]].view(og.ny, og.nx).cpu().numpy()
                gy = uyh[offs[i]:offs[i + 1]].view(og.ny, og.nx).cpu().numpy()
                dn = np.sqrt(((gx - oux)[fl_i] ** 2 + (gy - ouy)[fl_i] ** 2).sum())
                o_errs[i].append(float(dn / np.sqrt((oux[fl_i] ** 2 + ouy[fl_i] ** 2).sum())))
            o_secs += time.perf_counter() - o0
        ucells = lat_h.cells
        steady_ms = float(np.mean(cyc_ms[1:])) if len(cyc_ms) > 1 else cyc_ms[0]
        unsteady = {
            "workload": f"{len(ub)} flow-past-disk trajectories, sizes 128x128 / 256x128 / "
                        f"256x256 / 512x256 ({ucells} cells), tau U(0.55, 0.8), Re 50-200 on the "
                        f"channel height, cycle = {k_lbm} LBM steps + {m_fno} FNO steps "
                        f"(Delta T = {dT} Delta t) + reinit, CUDA graph per cycle",
            "cycles": args.unsteady_cycles, "cycle_ms": cyc_ms, "first_cycle_includes_capture": True,
            "cycle_ms_steady": steady_ms,
            "lbm_glups": k_lbm * ucells / (steady_ms * 1e-3) / 1e9,
            "rel_l2_u_vs_fp64_oracle_hybrid_per_cycle": {
                f"traj{i}_{ub[i]['nx']}x{ub[i]['ny']}": o_errs[i] for i in sample},
            "oracle_hybrid_seconds": o_secs,
            "pure_lbm_ms_per_cycle": float(np.mean(ref_ms)),
            "cost_ratio_vs_pure_lbm_same_time": steady_ms / float(np.mean(ref_ms)),
            "eps_N": 1.0 - k_lbm / (k_lbm + m_fno * dT),
            "rel_l2_u_vs_pure_lbm_per_cycle": errs,
            "reference": "parity: the FP64 oracle hybrid (same bfloat16 weights) on the two "
                         "smallest trajectories; cost: pure GPU LBM over the same physical time",
            "fno": "seeded random weights: the hybrid is ~100% off pure LBM in u, so the cost "
                   "ratio is launch-pattern arithmetic, not a speed-up at equal accuracy"}
        hyb_u.close()
        lat_h.close()
        lat_r.close()

    # double shear layer (Sec. 3.2): periodic 128^2, 100 trajectories, the 2.6 M model group
    # (density net on rho - 1: 14 channels, 3 layers, 8 modes; velocity net on (u, v): 14
    # channels, 3 layers, 32 modes; decoders 1 x 32; padding 9), random weights.  Hybrids
    # 1:k = one FNO step of Delta T = 223 LBM steps, then k Delta T of LBM, against pure
    # LBM over the same physical time; and the pure autoregressive FNO rollout.
    shear = None
    if rank == 0 and args.shear_trajectories > 0:
        import synth
        setup = synth.DoubleShear()
        ns, Ts, dT = setup.n, args.shear_trajectories, setup.steps_per_dT
        ics = synth.double_shear(Ts, seed=2000)
        s_fields = [torch.from_numpy(np.concatenate([ic[k].ravel() for ic in ics])).cuda()
                    for k in ("rho", "ux", "uy")]
        s_grids = [GridSpec(ns, ns, setup.tau)] * Ts
        s_masks = [np.zeros((ns, ns), bool)] * Ts
        d_s = synth.FnoShape(c_in=1, c_out=1, width=14, layers=3, modes=8, dec_size=32, padding=9)
        v_s = synth.FnoShape(c_in=2, c_out=2, width=14, layers=3, modes=32, dec_size=32,
                             padding=9)
        nparams = [int(sum(int(np.prod(sh)) for _, sh in synth.fno_param_shapes(x)))
                   for x in (d_s, v_s)]
        dnet = Fno(FnoShape(c_in=1, c_out=1, width=14, layers=3, modes=8, dec_size=32, padding=9),
                   synth.fno_flatten_params(d_s, synth.fno_random_params(d_s, seed=31,
                                                                         out_scale=1e-2)))
        vnet = Fno(FnoShape(c_in=2, c_out=2, width=14, layers=3, modes=32, dec_size=32,
                            padding=9),
                   synth.fno_flatten_params(v_s, synth.fno_random_params(v_s, seed=32,
                                                                         out_scale=1e-2)))

        def s_metrics(lat_a, lat_b):
            ra, ua, va = lat_a.macro()
            rb, ub, vb = lat_b.macro()
            mse = float(((ra - rb) ** 2 + (ua - ub) ** 2 + (va - vb) ** 2).mean() / 3.0)
            wa = lat_a.vorticity(ua, va).view(Ts, -1)
            wb = lat_b.vorticity(ub, vb).view(Ts, -1)
            ew = float(((wa - wb).norm(dim=1) / wb.norm(dim=1)).mean())
            return mse, ew

        arms = {}
        for label, k in (("1:1", 1), ("1:2", 2), ("1:3", 3), ("fno_only", 0)):
            cyc = 30 if k == 0 else -(-30 // (k + 1))
            lat_h = Lattice(s_grids, s_masks, u_max=0.3)
            lat_r = Lattice(s_grids, s_masks, u_max=0.3)
            lat_h.reinit(*s_fields, neq_mode=1)
            lat_r.reinit(*s_fields, neq_mode=1)
            hyb_s = Hybrid(lat_h, dnet, HybridConfig(mode=1, k_lbm=k * dT, m_fno=1, neq_mode=1,
                                                     in_channels=1, in_channels_u=6), fno_u=vnet)
            hms, rms_, mses, ews = [], [], [], []
            for _ in range(cyc):
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                hyb_s.advance(cycles=1)
                c1.record(stream)
                r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                r0.record(stream)
                lat_r.step((k + 1) * dT)
                r1.record(stream)
                torch.cuda.synchronize()
                hms.append(c0.elapsed_time(c1))
                rms_.append(r0.elapsed_time(r1))
                m_, w_ = s_metrics(lat_h, lat_r)
                mses.append(m_)
                ews.append(w_)
            steady_h = float(np.mean(hms[1:])) if cyc > 1 else hms[0]
            arms[label] = {"cycles": cyc, "lbm_steps_per_cycle": k * dT,
                           "cycle_ms": steady_h, "pure_lbm_ms_same_time": float(np.mean(rms_)),
                           "eps_T": 1.0 - steady_h / float(np.mean(rms_)),
                           "eps_N": 1.0 - k / (k + 1.0),
                           "mse_per_cycle": mses, "vorticity_rel_l2_per_cycle": ews,
                           "mse_global": float(np.mean(mses)),
                           "vorticity_global": float(np.mean(ews))}
            hyb_s.close()
            lat_h.close()
            lat_r.close()
        for label in ("1:1", "1:2", "1:3"):
            for key in ("mse_global", "vorticity_global"):
                base = arms["fno_only"][key]
                arms[label][key.replace("_global", "_reduction_vs_fno")] = (
                    (base - arms[label][key]) / base if base > 0 else None)
        shear = {"workload": f"double shear layer, {Ts} trajectories of {ns}x{ns} periodic, "
                             f"tau {setup.tau:.4f}, U {setup.u_lattice:.4f} (lattice), A1, A2 "
                             f"U(20, 125), Delta T = {dT} steps, 30 Delta T horizon",
                 "model_group": {"density_params": nparams[0], "velocity_params": nparams[1],
                                 "padding": 9,
                                 "path": ("tensor cores (14 channels zero-padded to 16, "
                                          f"{ns + 9} x {ns + 9} padded grid in "
                                          f"{(ns + 9 + 7) // 8 * 8} x {(ns + 9 + 63) // 64 * 64} "
                                          "storage)"
                                          if dnet.uses_tensor_cores(ns, ns) and
                                          vnet.uses_tensor_cores(ns, ns) else "CUDA cores")},
                 "arms": arms,
                 "fno": "seeded random weights: errors are not an accuracy claim"}
        dnet.close()
        vnet.close()

    # differentiable hybrid training step (rank 0): batch 8 porous 512 x 512, FNO 4 x 64
    # channels, 13 x 13 modes (11.1 M parameters, FP32 master weights), loss = MSE of
    # (rho, u) after 32 LBM steps that follow the FNO-based reinit, backward through the
    # LBM adjoint with f checkpointed every 8 steps, then an Adam update
    training = None
    if rank == 0 and args.train_steps > 0:
        import synth
        from paper_2604_27158_gb300.train import hybrid_loss
        Bt, Nt = 8, 512
        tshape_s = synth.FnoShape(c_in=4, c_out=3, width=64, layers=4, modes=13, dec_layers=1,
                                  dec_size=64)
        tshape = FnoShape(c_in=4, c_out=3, width=64, layers=4, modes=13, dec_layers=1,
                          dec_size=64)
        tparams = torch.nn.Parameter(torch.from_numpy(synth.fno_flatten_params(
            tshape_s, synth.fno_random_params(tshape_s, seed=5, out_scale=1e-2))
            .astype(np.float32)).cuda())
        tmasks = [synth.porous_media(Nt, Nt, 4, 12, seed=300 + k)[0] for k in range(Bt)]
        lat_t = Lattice([GridSpec(Nt, Nt, TAU, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                                  west_value=RHO_IN, east_value=RHO_OUT)] * Bt, tmasks)
        xt = torch.zeros((Bt, 4, Nt, Nt), device="cuda")
        xt[:, 3] = torch.from_numpy(np.stack(tmasks).astype(np.float32)).cuda()
        tgt = [torch.from_numpy(np.concatenate([np.asarray(synth.smooth_macro_fields(
            Nt, Nt, seed=400 + k, drho=1e-3, umax=0.02)[c]).ravel() for k in range(Bt)])).cuda()
            for c in range(3)]
        fluid_t = torch.from_numpy(~np.concatenate([m.ravel() for m in tmasks])).cuda()
        opt = torch.optim.Adam([tparams], lr=1e-4)

        def train_step():
            opt.zero_grad(set_to_none=True)
            loss = hybrid_loss(lat_t, tshape, tparams, xt, 32, tgt, every=8, fluid=fluid_t)
            loss.backward()
            opt.step()
            return loss

        for _ in range(2):
            train_step()
        torch.cuda.synchronize()
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        tl = []
        for _ in range(args.train_steps):
            tl.append(train_step())
        t1e.record(stream)
        torch.cuda.synchronize()
        tms = t0e.elapsed_time(t1e) / args.train_steps
        training = {
            "workload": "differentiable hybrid training step: batch 8 porous 512x512, FNO 4 "
                        "layers x 64 channels, 13x13 modes, decoder 64 -> 3 (FP32 master "
                        "weights), reinit, 32 LBM steps, MSE of (rho, u), backward through the "
                        "LBM adjoint (checkpoints every 8 steps) and the FNO adjoint, Adam",
            "params": int(tparams.numel()), "ms_per_step": tms,
            "samples_per_s": Bt / (tms * 1e-3),
            "loss_first_last": [float(tl[0]), float(tl[-1])],
            "gradient_check": "tests/test_gpu_train.py, tests/test_gpu_adjoint.py (FP64 "
                              "autograd references pinned to central differences)"}
        lat_t.close()
        del lat_t, tparams, opt

    # end to end through the public API with host buffers (pinned): masks in, fields out
    e2e = None
    if args.steps > 0:
        words = np.concatenate([P.pack_mask(m) for m in masks]).view(np.int32)
        mask_h = torch.from_numpy(words).pin_memory()
        out_h = torch.empty((3, cells), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_upd = 0
        for _ in range(args.steps):
            lat.mask.copy_(mask_h, non_blocking=True)
            est, _, _ = hyb.advance()
            rho_d, ux_d, uy_d = lat.macro()
            out_h[0].copy_(rho_d, non_blocking=True)
            out_h[1].copy_(ux_d, non_blocking=True)
            out_h[2].copy_(uy_d, non_blocking=True)
            torch.cuda.synchronize()
            e_upd += int(est.steps) * cells
        e_s = time.perf_counter() - t0
        e2e = {"value": e_upd / e_s / 1e9 * (world if world > 1 else 1), "unit": "GLUPS",
               "h2d_bytes_per_step": int(words.nbytes), "d2h_bytes_per_step": int(out_h.numel() * 4)}

    line = None
    if rank == 0:
        cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(masks)
        steps_per_solve = int(st.steps)
        line = {
            "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(T, phis, args.solve_steps, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "k_step_tma", "bytes_per_launch": BYTES_PER_CELL * cells,
                         "tile_shape": {"rows_per_tile": shape[1], "stages": shape[2],
                                        "ctas_per_sm": shape[3], "autotune_ms": tune_ms},
                         "launch_ms": kms, "traffic": step_kernel_traffic(cells, shape),
                         "traffic_unit": "bytes per launch (ncu dram read + write)"},
            "reinit_kernel": reinit_kernel,
            "time_to_steady_summary": None if tts is None else {
                "tol": tts["tol"], "trajectories": tts["trajectories"],
                "fno_init_s": tts["fno_init"]["seconds"],
                "fno_init_converged": tts["fno_init"]["converged"],
                "plain_init_s": tts["plain_init"]["seconds"],
                "plain_init_converged": tts["plain_init"]["converged"],
                "step_cap": tts["step_cap"]},
            "solve": {"lbm_steps": steps_per_solve, "converged": bool(st.converged),
                      "max_residual": float(st.max_residual)},
            "time_to_steady": tts,
            "tolerance_ladder": ladder,
            "lbm_sweep": sweep,
            "launch_bound": launch_bound,
            "hybrid_training": training,
            "double_shear": shear,
            "fno_throughput": fno_tp,
            "unsteady_hybrid": unsteady,
            "gpu_launches": None,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        # our kernels per step: FNO on the tensor-core path (table kernel + lift + 5 per
        # layer + decoder, else 2 twiddle + lift + 5 per layer + decoder), reinit, fill,
        # pack/unpack, one step kernel per LBM step (a check runs the step kernel with
        # statistics: the last check's step is computed and not kept), two reduction
        # kernels per check
        fno_k = (1 + 1 + 5 * 4 + 1) if net.uses_tensor_cores(NY, NX) else (2 + 1 + 5 * 4 + 1)
        per_step = (fno_k + 1 + 1 + 2 + steps_per_solve + 1
                    + 2 * math.ceil(steps_per_solve / CHECK_EVERY))
        line["gpu_launches"] = per_step * args.steps
        print(json.dumps(line), flush=True)
    hyb.close()
    lat.close()
    net.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
