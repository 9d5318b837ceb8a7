#!/usr/bin/env python3
"""Benchmark: BSSN moving-puncture evolution, RK4 method of lines, on GB300.

Workload (default): single Brill-Lindquist puncture, M = 1, on a 128^3 grid
over [-8, 8]^3 (puncture half a cell off every grid point), W variable, 1+log
slicing, Gamma-driver shift with eta = 2/M, Sommerfeld outer boundary, three
ghost layers, RK4 with dt = 0.25 h, float64.  One "step" is one full RK4 step
(four fused right-hand-side stages plus the boundary) over the whole grid.
Throughput is reported as interior point-updates per second (one point
advanced one RK4 step).

Launch: ``python bench.py [--gpus N] [--steps K] [--warmup W]`` for N = 1, or
under torchrun for N > 1 (one independent replica per GPU: the path does not
shard, so ranks exchange nothing but the timing barrier).
``--impl reference`` times the CPU oracle (plain float64 C) on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 128
DOMAIN = 8.0
# Float64 work per interior point per fused stage launch (right-hand side plus
# RK4 combine), from the ncu instruction counts of the stage kernel
# (profiles/stage_fp64_bl64.md): 535 DADD + 239 DMUL + 1485 DFMA.
FLOP_PER_POINT_RHS = 3744.0        # DADD + DMUL + 2 DFMA
DPINST_PER_POINT_RHS = 2259.0      # float64 instructions issued
# The 32-wide tiles on grids whose n0 is a multiple of 32 and whose n1, n2
# fill the blocks (the benchmark grid) run the full-block kernel: x-mixed
# second differences shared across lanes, D_y D_z across rows through shared
# memory; 302.5 DADD + 251.8 DMUL + 1366.8 DFMA per point
# (profiles/stage_fp64_rows_bl64.md).
ROWS_TILES = ("32x8x1/1", "32x4x1/1", "32x4x2/1", "32x2x2/2")
FLOP_PER_POINT_RHS_ROWS = 3287.9
DPINST_PER_POINT_RHS_ROWS = 1921.1
HBM_BYTES_PER_POINT_STEP = 3264.0  # 17 register passes x 24 fields x 8 B
# mixed: float stage buffers (24 x 4 B) each with a float64 W (8 B), 104 B a
# buffer pass; per RK4 step: stage 1 reads m0, writes m1 and the k-sum (312 B);
# stages 2-3 read src, m0 and the k-sum and write out and the k-sum (520 B
# each); stage 4 reads src and the k-sum, reads and writes y_n (2 x 192 B) and
# writes the new shadow m0 (696 B)
HBM_BYTES_PER_POINT_STEP_MIXED = 312.0 + 2 * 520.0 + 696.0   # 2048
def _measured_hbm_gbs(default=6764.0):
    """The STREAM-style copy bandwidth measured on these GB300s
    (MEASURED_PEAKS.json beside this file, key hbm_gbs); the value it held
    when the file is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return default


HBM_MEASURED_GBS = _measured_hbm_gbs()
FP64_PEAK_GFLOPS = 1250.0          # nominal GB300 FP64 rate
FP64_MEASURED_GFLOPS = 1196.0      # dependent-chain DFMA microbenchmark on GB300 (2070 MHz)
# DRAM bytes (read + write) per interior point of one stage launch, from the
# ncu capture of the current kernels on the 64^3 case (traffic grows with the
# points; profiles/stage_traffic_bl64.md); None until captured.
FP64_TRAFFIC_PER_POINT = 1587.9    # (100.8 + 315.4) MB / 262,144 points, stage_fp64_kernel 64x4x1/1
FP64_ROWS_TRAFFIC_PER_POINT = 620.3  # (83.2 + 79.4) MB / 262,144 points, stage_fp64_blocks_kernel 32x4x1/1
MIXED_TRAFFIC_PER_POINT = 488.0    # mean over the 4 stages of stage_mixed_tma_kernel: 282, 501, 492, 677 B
# Float64 work per interior point of the analysis kernels (DADD + DMUL + 2 DFMA
# from ncu instruction counts; profiles/analysis_kernels_bl96.md).
# psi4 and constraints include the ADM-field pass that precedes them
# (36 flop per stored point, 44 per interior point at 96^3).
ANALYSIS_FLOP_PER_POINT = {"psi4": 3409.0 + 44.0, "adm_integrals": 1771.9, "constraints": 1999.0 + 44.0}


def workload_params(precision="fp64"):
    from paper_1111_3344_gb300.bssn import Params
    h = 2 * DOMAIN / N_SIDE
    # mixed: W right-hand side in float64 below W = 0.2 (r < ~0.6 M from the puncture)
    return Params(n=(N_SIDE,) * 3, xmin=(-DOMAIN,) * 3, h=h, boundary="sommerfeld", conformal="W",
                  slicing="1+log", shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * h,
                  precision=precision, w_fp64_threshold=0.2, r_excise=1.0)


BL_P = [1, 1.0, 0.0, 0.0, 0.0]


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n_gpus:
        raise SystemExit(f"--gpus {n_gpus} but WORLD_SIZE={world}")
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def max_over_ranks(x, world):
    """Max of a per-rank scalar over all ranks (the timing barrier's reduction;
    the evolutions themselves exchange nothing)."""
    import torch
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank, steps, ms_local, world):
    """Whole-job point-updates/s (millions): every rank advances its own replica
    of the workload; the job takes as long as the slowest rank."""
    ms = max_over_ranks(ms_local, world)
    return points_per_rank * steps * world / (ms * 1e-3) / 1e6, ms


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name, or implementer/part
    on Arm), with the machine type."""
    import platform
    name = ""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "Model", "CPU part"):
            vals = [ln.split(":", 1)[1].strip() for ln in info if ln.lower().startswith(key.lower())]
            if vals:
                name = f"{key} {vals[0]}"
                break
    except OSError:
        pass
    return f"{platform.machine()} {name}".strip()


def oracle_cpu_baseline(min_s=10.0, max_steps=12):
    """The float64 CPU oracle on full RK4 steps of the same workload: as many
    as fit in about min_s seconds (at least one, at most max_steps)."""
    import oracle as O
    cfg = O.Config(n=(N_SIDE,) * 3, xmin=(-DOMAIN,) * 3, h=2 * DOMAIN / N_SIDE, periodic=False,
                   use_w=True, slicing="1+log", shift="gamma-driver", eta=2.0, ko_eps=0.1,
                   dt=0.25 * 2 * DOMAIN / N_SIDE, punctures=[(1.0, 0.0, 0.0, 0.0)])
    st = O.initial_data(cfg, "bl", BL_P)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < min_s):
        st = O.rk4(cfg, st, 1)
        steps += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N_SIDE ** 3 * steps / dt / 1e6, "unit": "Mpoint-updates/s", "cores": cores,
            "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{steps} full RK4 steps of the {N_SIDE}^3 puncture workload ({dt:.1f} s)"}


def run_reference(args):
    """--impl reference: the CPU oracle, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    cfg = O.Config(n=(N_SIDE,) * 3, xmin=(-DOMAIN,) * 3, h=2 * DOMAIN / N_SIDE, periodic=False,
                   use_w=True, slicing="1+log", shift="gamma-driver", eta=2.0, ko_eps=0.1,
                   dt=0.25 * 2 * DOMAIN / N_SIDE, punctures=[(1.0, 0.0, 0.0, 0.0)])
    st = O.initial_data(cfg, "bl", BL_P)
    rng = np.random.default_rng(0)
    npts = 8192
    ijk = np.stack([rng.integers(3, 3 + N_SIDE, npts) for _ in range(3)], axis=1).astype(np.int32)
    for _ in range(args.warmup):
        O.rhs_points(cfg, st, ijk)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(4):  # four right-hand sides per RK4 point-update
            O.rhs_points(cfg, st, ijk)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = npts * args.steps / tot / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "metric": "BSSN RK4 point-updates/s (FP64, Brill-Lindquist puncture 128^3)",
        "value": value, "unit": "Mpoint-updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": "single Brill-Lindquist puncture M=1, 128^3 on [-8,8]^3, W, 1+log, "
                               "Gamma-driver eta=2, Sommerfeld, RK4 dt=0.25h",
                   "sample": f"{npts} random interior points x 4 right-hand sides per step"},
        "cpu_baseline": {"value": value, "unit": "Mpoint-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{npts} random interior points x 4 right-hand sides per step"},
        "e2e": {"value": value, "unit": "Mpoint-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args):
    import torch

    from paper_1111_3344_gb300 import bssn as B
    rank, world, local = dist_setup(args.gpus)
    params = workload_params(args.precision)
    evo = B.Evolution(params)
    evo.set_initial_data("bl", BL_P)
    stream = evo.stream
    if args.tile:  # a fixed configuration (profiling captures)
        tile = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())].index(args.tile)
        B.bssn_set_tile(evo.ctx, tile)
    else:
        tile, tile_ms = B.bssn_autotune(evo.ctx, reps=5)  # untimed: picks the stage-kernel tiles
    for _ in range(args.warmup):
        evo.rk4_step(1)
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    B.bssn_profile(evo.ctx, True)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    barrier(world)
    start.record(stream)
    for _ in range(args.steps):
        evo.rk4_step(1)
    stop.record(stream)
    stop.synchronize()
    barrier(world)
    ms_local = start.elapsed_time(stop)
    stage_ms, stage_n, bc_ms, bc_n = B.bssn_profile(evo.ctx, False)
    clk = clocks.stop()
    pts = N_SIDE ** 3
    value, ms = whole_job_rate(pts, args.steps, ms_local, world)

    # end to end through the C ABI with pinned host buffers: upload state,
    # one RK4 step, read the state back, every step
    host_in = torch.empty(evo.shape, dtype=torch.float64, pin_memory=True).numpy()
    # two read-back buffers: the copy of step n's state to the host runs on
    # the library's copy stream while step n+1's state is uploaded
    host_out = [torch.empty(evo.shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    host_in[...], _ = evo.get_state()
    evo.enable_copy_staging()  # the copies overlap the steps as well as each other
    e2e_steps = max(2, args.steps)
    barrier(world)
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        B.bssn_set_state_async(evo.ctx, host_in, 0.0)
        evo.rk4_step(1)
        B.bssn_get_state_async(evo.ctx, host_out[s % 2])
    B.bssn_wait_state(evo.ctx)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = pts * e2e_steps * world / e2e_s / 1e6
    nbytes = host_in.nbytes

    rows = B.bssn_tile_name(tile) in ROWS_TILES and N_SIDE % 32 == 0
    flop_pt = FLOP_PER_POINT_RHS_ROWS if rows else FLOP_PER_POINT_RHS
    dpinst_pt = DPINST_PER_POINT_RHS_ROWS if rows else DPINST_PER_POINT_RHS
    traffic_pt = FP64_ROWS_TRAFFIC_PER_POINT if rows else FP64_TRAFFIC_PER_POINT
    flop_launch = flop_pt * pts
    stage_launch_ms = stage_ms / max(stage_n, 1)
    achieved = flop_launch / (stage_launch_ms * 1e-3) / 1e12
    mixed = args.precision == "mixed"
    if mixed:
        # HBM-bound form: algorithmic bytes per stage launch over its duration
        bytes_launch = HBM_BYTES_PER_POINT_STEP_MIXED / 4.0 * pts
        gbs = bytes_launch / (stage_launch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": B.bssn_tile_name(tile), "achieved": gbs,
                    "peak": HBM_MEASURED_GBS, "unit": "GB/s", "frac": gbs / HBM_MEASURED_GBS,
                    "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                    "algorithmic_bytes_per_launch": bytes_launch,
                    "traffic": MIXED_TRAFFIC_PER_POINT * pts if MIXED_TRAFFIC_PER_POINT else None,
                    "launch_ms": stage_launch_ms, "launches": stage_n,
                    "boundary_launch_ms": bc_ms / max(bc_n, 1)}
    else:
        roofline = {"bound": "alu", "kernel": "stage_fp64_blocks_kernel" if rows else "stage_fp64_kernel",
                    "achieved": achieved * 1e3,
                    "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)",
                    "peak_source": "nominal GB300 FP64 rate (no tensor-core path: stencil)",
                    "frac": achieved * 1e3 / FP64_PEAK_GFLOPS,
                    "frac_of_measured_dfma": achieved * 1e3 / FP64_MEASURED_GFLOPS,
                    "fp64_issue_frac": dpinst_pt * pts / (stage_launch_ms * 1e-3)
                                       / (FP64_MEASURED_GFLOPS * 1e9 / 2),
                    "traffic": traffic_pt * pts,
                    "launch_ms": stage_launch_ms, "launches": stage_n,
                    "boundary_launch_ms": bc_ms / max(bc_n, 1),
                    "hbm_frac": (HBM_BYTES_PER_POINT_STEP * pts * args.steps / (ms * 1e-3)) / HBM_MEASURED_GBS / 1e9}
    line = {
        "metric": ("BSSN RK4 point-updates/s (mixed FP32 RHS / FP64 state, Brill-Lindquist puncture 128^3)"
                   if mixed else "BSSN RK4 point-updates/s (FP64, Brill-Lindquist puncture 128^3)"),
        "value": value, "unit": "Mpoint-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": "single Brill-Lindquist puncture M=1, 128^3 on [-8,8]^3, W, 1+log, "
                               "Gamma-driver eta=2, Sommerfeld, RK4 dt=0.25h",
                   "global_batch": world, "grid": [N_SIDE] * 3, "parallelism": f"replicas{world}",
                   "precision": args.precision, "tile": B.bssn_tile_name(tile),
                   "l2": "inputs larger than L2 (4 float64 registers of 469 MB each)"},
        "roofline": roofline,
        "rhs_evaluations_per_s": 4.0 * value * 1e6,  # four right-hand sides per point-update
        "e2e": {"value": e2e_value, "unit": "Mpoint-updates/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
                "copies": "pinned; device staging areas: the upload of step n+1 and the read-back "
                          "of step n overlap each other and the steps"},
        # the split mixed stage is two kernels per stage (stencils, algebra)
        "gpu_launches": stage_n * (2 if B.bssn_tile_name(tile).startswith("split") else 1) + bc_n,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    evo.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _bl_params(member, precision):
    from paper_1111_3344_gb300.bssn import Params
    h = member["h"]
    return Params(n=member["n"], xmin=member["xmin"], h=h, boundary="sommerfeld", conformal="W",
                  slicing="1+log", shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * h,
                  precision=precision, w_fp64_threshold=0.2, r_excise=1.0)


def run_batched(args):
    """64 time-symmetric Brill-Lindquist binaries (masses U[0.3,0.7], separations
    U[2,6], grids from {48,64,96,128}^3, seed 1111) advanced together, one
    persistent launch per RK4 stage under a CUDA graph."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    from paper_1111_3344_gb300 import inputs
    torch.cuda.set_device(0)
    members = inputs.binary_bl_batch(seed=1111, count=args.members)
    params = [_bl_params(m, args.precision) for m in members]
    need = sum(B.Batch.member_bytes(p) for p in params) + (64 << 20)
    batch = B.Batch(args.precision, pool_bytes=need, max_members=max(len(params), 1))
    ids = []
    for m, p in zip(members, params):
        mid = batch.add(p)
        bl = [len(m["punctures"])] + [v for q in m["punctures"] for v in q]
        batch.set_initial_data(mid, "bl", bl)
        ids.append(mid)
    best, tile_ms = batch.autotune(reps=2)
    if args.tile:
        best = list(tile_ms).index(args.tile)
        batch.set_tile(best)
    batch.step(args.warmup)
    batch.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(batch.stream)
    batch.step(args.steps)
    stop.record(batch.stream)
    stop.synchronize()
    ms = start.elapsed_time(stop)
    pts = sum(p.n[0] * p.n[1] * p.n[2] for p in params)
    value = pts * args.steps / (ms * 1e-3) / 1e6
    # launches per step: a stage and a boundary launch per RK4 stage; the
    # one-block-per-tile float64 configurations launch the members with full
    # tiles and the others separately
    tname = list(tile_ms)[best]
    stage_launches = 1
    if tname.startswith("tiles") and args.precision == "fp64":
        tx, ty, tz = (int(v) for v in tname[len("tiles"):].split("/")[0].split("x"))
        full = [tx == 32 and p.n[0] % 32 == 0 and p.n[1] % ty == 0 and p.n[2] % tz == 0 for p in params]
        stage_launches = int(any(full)) + int(not all(full))
    line = {"metric": f"batched BSSN RK4 point-updates/s ({args.precision})", "value": value,
            "unit": "Mpoint-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": f"{len(params)} Brill-Lindquist binaries, grids {{48,64,96,128}}^3, seed 1111",
                       "interior_points": pts, "tile": list(tile_ms)[best],
                       "autotune_ms_stage1": {k: round(v, 3) for k, v in tile_ms.items() if v >= 0},
                       "launches_per_step": 4 * (stage_launches + 1), "graph": True}}
    print(json.dumps(line))
    batch.close()


def run_served(args):
    """Poisson arrivals of puncture evolutions (grids 32^3..192^3, 50..400 steps,
    Brill-Lindquist binaries as in the batched workload, seed 3344), admitted by
    HBM budget into a continuous-batching server; reports p50/p99 time from
    submission to completion and the aggregate point-update rate."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    torch.cuda.set_device(0)
    rng = np.random.default_rng(3344)
    sizes = [32, 48, 64, 96, 128, 160, 192]
    reqs = []
    for _ in range(args.requests):
        n = int(rng.choice(sizes))
        steps = int(rng.integers(50, 401))
        m1, m2 = rng.uniform(0.3, 0.7, size=2)
        sep = rng.uniform(2.0, 6.0)
        L = max(8.0, 2.0 * sep) * (m1 + m2)
        h = 2 * L / n
        x1, x2 = sep * m2 / (m1 + m2), -sep * m1 / (m1 + m2)
        x1 = -L + round((x1 + L) / h) * h
        x2 = -L + round((x2 + L) / h) * h
        mem = dict(n=(n, n, n), xmin=(-L,) * 3, h=h)
        reqs.append((_bl_params(mem, args.precision), [2, m1, x1, 0.0, 0.0, m2, x2, 0.0, 0.0], steps))
    work = sum(p.n[0] ** 3 * st for p, _, st in reqs)
    budget = int(args.budget_gb * (1 << 30))
    srv = B.Server(args.precision, budget_bytes=budget)
    # arrival rate: 0.8 x the capacity in requests/s implied by a throughput estimate
    est_rate = args.capacity_mpts * 1e6  # point-updates/s
    lam = 0.8 * est_rate / (work / len(reqs))
    gaps = rng.exponential(1.0 / lam, size=len(reqs))
    t0 = time.perf_counter()
    tickets = []
    for (p, idp, st), gap in zip(reqs, gaps):
        time.sleep(gap)
        tickets.append(srv.submit(p, "bl", idp, st))
    lats, fails = [], 0
    for t in tickets:
        st, norms, lat = srv.wait(t, timeout=3600)
        lats.append(lat)
        fails += st != 0
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lats = np.array(lats)
    line = {"metric": "served BSSN evolutions: p50/p99 completion latency, aggregate point-updates/s",
            "value": stats["point_updates"] / wall / 1e6, "unit": "Mpoint-updates/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "p50_s": float(np.percentile(lats, 50)), "p99_s": float(np.percentile(lats, 99)),
            "failed": int(fails), "wall_s": wall, "busy_s": stats["busy_s"],
            "config": {"workload": f"{len(reqs)} Poisson-arrival Brill-Lindquist binaries, grids 32^3..192^3, "
                                   f"50..400 steps, seed 3344", "precision": args.precision, "lambda_per_s": lam,
                       "budget_gb": args.budget_gb, "point_updates": work}}
    print(json.dumps(line))


def run_precision(args):
    """Mixed precision against float64 on the same GPU: the puncture at
    args.n^3 (256^3 by default for this mode) evolved args.steps RK4 steps
    both ways; per-field L2/Linf of the state difference, relative difference
    of every constraint norm, and the speedup."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    torch.cuda.set_device(0)
    out = {}
    for prec in ("fp64", "mixed"):
        evo = B.Evolution(workload_params(prec))
        evo.set_initial_data("bl", BL_P)
        B.bssn_autotune(evo.ctx, reps=2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        evo.rk4_step(args.steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st, _ = evo.get_state()
        out[prec] = (st, evo.constraints(), dt)
        evo.close()
        del evo
        torch.cuda.empty_cache()
    s64, c64, t64 = out["fp64"]
    smx, cmx, tmx = out["mixed"]
    g = 3
    d = (smx - s64)[:, g:-g, g:-g, g:-g].reshape(24, -1)
    ref = np.abs(s64[:, g:-g, g:-g, g:-g]).reshape(24, -1).max(axis=1)
    names = ["chi", "gt_xx", "gt_xy", "gt_xz", "gt_yy", "gt_yz", "gt_zz", "trK", "At_xx", "At_xy",
             "At_xz", "At_yy", "At_yz", "At_zz", "Gt_x", "Gt_y", "Gt_z", "alpha", "beta_x", "beta_y",
             "beta_z", "B_x", "B_y", "B_z"]
    fields = {nm: {"L2": float(np.sqrt((d[f] ** 2).mean())), "Linf": float(np.abs(d[f]).max()),
                   "max_abs_fp64": float(ref[f])} for f, nm in enumerate(names)}
    cn = ["H", "Mx", "My", "Mz"]
    keys = [f"{k}_{n}_{s}" for s in ("full", "excised") for k in ("L2", "Linf") for n in cn]
    rel = {k: float(abs(a - b) / abs(b)) if b != 0 else None for k, a, b in zip(keys, cmx, c64)}
    line = {"metric": "mixed vs float64: per-field state error and constraint-norm relative difference",
            "grid": args.n, "steps": args.steps, "speedup_mixed_over_fp64": t64 / tmx,
            "seconds": {"fp64": t64, "mixed": tmx}, "constraint_norms_fp64": dict(zip(keys, c64.tolist())),
            "constraint_norm_rel_diff": rel, "fields": fields}
    print(json.dumps(line))


def run_analysis(args):
    """The analysis steps after the evolution on the benchmark puncture:
    Weyl scalar Psi4, ADM mass / angular momentum volume integrals, constraint
    norms (all float64), each timed over K launches with CUDA events on the
    library's stream after W warm-up launches; the puncture tracker's cost
    per RK4 step (steps with and without tracking); and RK4 steps of the
    matter-coupled right-hand side (a smooth seeded T_{mu nu}) against vacuum."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    torch.cuda.set_device(0)
    evo = B.Evolution(workload_params("fp64"))
    evo.set_initial_data("bl", BL_P)
    B.bssn_autotune(evo.ctx, reps=2)
    evo.rk4_step(4)  # a state with shift, B and K away from their initial zeros
    pts = N_SIDE ** 3
    psi4_out = evo.psi4()
    stream = evo.stream
    kernels = {"psi4": lambda: evo.psi4(psi4_out), "adm_integrals": lambda: evo.adm_integrals(),
               "constraints": lambda: evo.constraints()}
    clocks = ClockSampler(0)
    clocks.start()
    res = {}
    for name, fn in kernels.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms": ms, "Mpoints_per_s": pts / ms / 1e3,
                     "fp64_gflops": ANALYSIS_FLOP_PER_POINT[name] * pts / (ms * 1e-3) / 1e9}
    # tracker: RK4 steps with and without it
    times = {}
    for track in (False, True):
        evo.set_punctures([(1.0, 0.0, 0.0, 0.0)])
        evo.track_punctures(track)
        evo.rk4_step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        evo.rk4_step(args.steps)
        e1.record(stream)
        e1.synchronize()
        times[track] = e0.elapsed_time(e1) / args.steps
    # matter-coupled right-hand side: RK4 steps with a smooth seeded T_{mu nu}
    # (10 more float64 fields read per point) against vacuum, same state
    from paper_1111_3344_gb300 import inputs
    evo.track_punctures(False)
    prm = workload_params("fp64")
    tmunu = inputs.random_tmunu(7, prm.n, prm.xmin, prm.h)
    mtimes = {}
    for matter in (False, True):
        evo.set_matter(tmunu if matter else None)
        evo.rk4_step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        evo.rk4_step(args.steps)
        e1.record(stream)
        e1.synchronize()
        mtimes[matter] = e0.elapsed_time(e1) / args.steps
    evo.set_matter(None)
    clk = clocks.stop()
    evo.close()
    top = res["psi4"]
    line = {
        "metric": "BSSN analysis point-evaluations/s (Psi4, Brill-Lindquist puncture 128^3)",
        "value": top["Mpoints_per_s"], "unit": "Mpoints/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": top["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "Psi4 / ADM integrals / constraint norms of the 128^3 puncture after 4 RK4 steps",
                   "grid": [N_SIDE] * 3},
        "roofline": {"bound": "alu", "kernel": "psi4_kernel", "achieved": top["fp64_gflops"],
                     "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s (FP64)",
                     "frac": top["fp64_gflops"] / FP64_PEAK_GFLOPS, "traffic": None},
        "kernels": res,
        "tracker": {"ms_per_step_without": times[False], "ms_per_step_with": times[True],
                    "overhead_ms": times[True] - times[False]},
        "matter": {"ms_per_step_vacuum": mtimes[False], "ms_per_step_with_tmunu": mtimes[True],
                   "Mpoint_updates_per_s_with_tmunu": pts / mtimes[True] / 1e3},
        "gpu_launches": 3 * args.steps + 2 * args.steps * (1 + 8) + 2 * args.steps * 8,
        "clocks": clk,
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default=None,
                    help="default: mixed for the served workload (its configuration), float64 otherwise")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["puncture", "batched", "served", "precision", "analysis"],
                    default="puncture",
                    help="puncture: the benchmark line (single 128^3 puncture); batched / served: "
                         "the multi-evolution workloads, reported on their own lines")
    ap.add_argument("--tile", default=None, help="stage-kernel configuration name (default: autotune)")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--capacity-mpts", type=float, default=None,
                    help="served: throughput estimate (M point-updates/s) that sets the arrival rate "
                         "(default 250 mixed, 50 float64)")
    ap.add_argument("--n", type=int, default=128,
                    help="grid points per side (128 is the benchmark workload; smaller sizes are "
                         "for profiling captures only)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "mixed" if args.workload == "served" else "fp64"
    if args.capacity_mpts is None:
        args.capacity_mpts = 250.0 if args.precision == "mixed" else 50.0
    global N_SIDE
    N_SIDE = args.n
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "analysis":
        run_analysis(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
