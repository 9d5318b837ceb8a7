#!/usr/bin/env python3
"""Benchmark: BSSN moving-puncture evolution, RK4 method of lines, on GB300.

Workload (default): single Brill-Lindquist puncture, M = 1, on a 128^3 grid
over [-8, 8]^3 (puncture half a cell off every grid point), W variable, 1+log
slicing, Gamma-driver shift with eta = 2/M, Sommerfeld outer boundary, three
ghost layers, RK4 with dt = 0.25 h, float64.  One "step" is one full RK4 step
(four fused right-hand-side stages plus the boundary) over the whole grid.
Throughput is reported as interior point-updates per second (one point
advanced one RK4 step).

At N = 1 the same line also carries the rest of the benchmark's metric, each
part timed with its own CUDA events and clock sample: ``mixed`` (the same
puncture with float32 stencils and right-hand side, float64 RK4 state),
``batched`` (64 Brill-Lindquist binaries on grids 48^3..128^3, float64,
mixed and double-word, a few of their 100 steps) and ``served_sample`` (the
first requests of the served workload's Poisson stream at 0.8x a capacity
measured in the same run, with p50/p99 completion latency; the server steps
the shortest remaining work first, at least 2^21 interior points per step,
unless ``--serve-policy all``).

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
# Algorithmic HBM bytes per interior point-update (one RK4 step; every
# register read or written once per pass, 24 fields): float64 3072 B -- stage
# 1 reads y_n and writes the stage value and k-sum (576), stages 2 and 3 read
# the stage value, y_n and the k-sum and write the next stage value and the
# k-sum (960 each), stage 4 reads the stage value and the k-sum and writes
# y_n (576); mixed 2496 B, the stage values in float (480 + 768 + 768 + 480).
# The dominant kernel's roofline uses the mean per stage launch (a quarter).
# The double-word path moves 8-byte values like float64 but also reads y_n and
# writes its double-word shadow in stage 4 (576 + 960 + 960 + 960 = 3456 B).
ALG_BYTES_PER_POINT_STEP = {"fp64": 3072.0, "mixed": 2496.0, "ff": 3456.0}
# Float64 work the stage kernels execute per interior point per launch
# (right-hand side plus RK4 combine), from ncu instruction counts at 64^3
# (DADD + DMUL + 2 DFMA): the every-stencil kernel 535 DADD + 239 DMUL + 1485
# DFMA; the full-block kernel (32-wide rows, D_y D_z through shared memory)
# 299.5 DADD + 246.8 DMUL + 1359.8 DFMA (per warp of 32 points, 1934 warp
# instructions issued to the float64 pipe).
FLOP_PER_POINT_RHS = 3744.0
DPINST_PER_POINT_RHS = 2259.0
ROWS_TILES = ("32x8x1/1", "32x4x1/1", "32x4x2/1", "32x2x2/2")
FLOP_PER_POINT_RHS_ROWS = 3265.8
DPINST_PER_POINT_RHS_ROWS = 1906.0
# Operations of one right-hand side at an interior point in the oracle's
# printed arrangement (its instrumented build, W variant, Gamma-driver shift:
# 5395 additions, 7874 multiplications, 299 divisions).  The arrangement
# evaluates all 81 second derivatives of gt_ij, symmetric duplicates
# included, as 25-point products, so it is 4.1x the kernels' count: it is
# reported beside the roofline, not used as its numerator.
ORACLE_FLOP_PER_POINT_RHS = 5395 + 7874 + 299
# DRAM bytes (read + write) per interior point of one stage launch, the mean
# over the four stages of one RK4 step, from ncu captures of single launches
# at the benchmark size (TRAFFIC_N^3; dram__bytes_read.sum +
# dram__bytes_write.sum), by stage-kernel configuration; a configuration
# without a capture of its current kernel, or a run at another grid size
# (where the share of ghosts, padding and L2 hits differs), reports null.
TRAFFIC_N = 128
STAGE_TRAFFIC_PER_POINT = {
    ("fp64", "32x4x1/1"): 937.2,       # stage_fp64_blocks_kernel: 7861.6 MB per step
    ("mixed", "tma32x4x1/2"): 565.3,   # stage_mixed_tma_kernel, 8 staged fields: 4741.9 MB per step
    ("mixed", "tma11_32x8x1/1"): 565.4,  # stage_mixed_tma_kernel, 11 staged fields: 4742.4 MB per step
}
# Float64 work per interior point of the analysis kernels (DADD + DMUL + 2 DFMA
# from ncu instruction counts at 96^3).  psi4 and constraints include the
# ADM-field pass that precedes them (36 flop per stored point, 44 per
# interior point at 96^3).
ANALYSIS_FLOP_PER_POINT = {"psi4": 3409.0 + 44.0, "adm_integrals": 1771.9, "constraints": 1999.0 + 44.0}


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
FP64_NOMINAL_GFLOPS = 1250.0        # nominal GB300 float64 rate (context only)


def workload_params(precision="fp64"):
    """The benchmark puncture's parameters in one precision form: fp64, mixed,
    mixed_ks64 (mixed with the k-sum of every field in float64) or ff
    (double-word right-hand side)."""
    from paper_1111_3344_gb300.bssn import Params
    h = 2 * DOMAIN / N_SIDE
    ks64 = precision == "mixed_ks64"
    # mixed: W right-hand side in float64 below W = 0.2 (r < ~0.6 M from the puncture)
    return Params(n=(N_SIDE,) * 3, xmin=(-DOMAIN,) * 3, h=h, boundary="sommerfeld", conformal="W",
                  slicing="1+log", shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * h,
                  precision="mixed" if ks64 else precision, ksum_fp64=ks64, w_fp64_threshold=0.2,
                  r_excise=1.0)


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


def _sink(torch):
    return torch.zeros(1, dtype=torch.float64, device="cuda")


def measured_peaks(B, torch, stream):
    """float64 and float32 multiply-add rates of this GPU, GFLOP/s, measured in
    this process by the library's probe (bssn_peak_probe)."""
    sink = _sink(torch)
    with torch.cuda.stream(stream):
        fp64 = B.bssn_peak_probe("fp64", sink.data_ptr(), stream.cuda_stream, reps=5)
        fp32 = B.bssn_peak_probe("fp32", sink.data_ptr(), stream.cuda_stream, reps=5)
    return {"fp64_gflops": fp64, "fp32_gflops": fp32,
            "how": "bssn_peak_probe: 152x4 blocks x 256 threads x 8 independent FMA chains, CUDA events, "
                   "2 flops per FMA, measured in this run"}


def confirm_by_steps(tile_ms, set_cfg, step, stream, top=3, steps=1):
    """The autotuners time the first two RK4 stages (the state stays unchanged);
    a configuration's last stage, which advances y_n, can weigh differently.
    Time `steps` whole RK4 steps under each of the `top` fastest candidates
    (CUDA events on the stream the steps run on, after one untimed step under
    that configuration) and keep the fastest.  Returns (index, {name: ms per
    step}).  The state advances: call before the warm-up."""
    import torch
    names = list(tile_ms)
    cands = sorted((c for c, nm in enumerate(names) if tile_ms[nm] >= 0), key=lambda c: tile_ms[names[c]])[:top]
    ms_step = {}
    for c in cands:
        set_cfg(c)
        step(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(steps)
        e1.record(stream)
        e1.synchronize()
        ms_step[names[c]] = e0.elapsed_time(e1) / steps
    best = min(cands, key=lambda c: ms_step[names[c]])
    set_cfg(best)
    return best, ms_step


def puncture_run(args, precision, world, local, steps, e2e=True):
    """The single-puncture workload at N_SIDE^3 in one precision: autotuned
    tiles, W untimed warm-up steps, then `steps` RK4 steps timed with CUDA
    events on the library's stream (clocks sampled meanwhile), with the stage
    and boundary launch durations; then `steps` end-to-end steps through the
    C ABI with the state uploaded from and read back to pinned host memory
    every step."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    params = workload_params(precision)
    evo = B.Evolution(params)
    evo.set_initial_data("bl", BL_P)
    stream = evo.stream
    if args.tile:  # a fixed configuration (profiling captures)
        tile = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())].index(args.tile)
        B.bssn_set_tile(evo.ctx, tile)
    else:
        # untimed: the autotuner's two-stage timing, then whole steps of its
        # three fastest candidates
        _, tile_ms = B.bssn_autotune(evo.ctx, reps=5)
        tile, _ = confirm_by_steps(tile_ms, lambda c: B.bssn_set_tile(evo.ctx, c), evo.rk4_step, stream,
                                   steps=2)
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
    for _ in range(steps):
        evo.rk4_step(1)
    stop.record(stream)
    stop.synchronize()
    barrier(world)
    ms_local = start.elapsed_time(stop)
    stage_ms, stage_n, bc_ms, bc_n = B.bssn_profile(evo.ctx, False)
    clk = clocks.stop()
    pts = N_SIDE ** 3
    value, ms = whole_job_rate(pts, steps, ms_local, world)
    out = {"value": value, "ms": ms, "steps": steps, "tile": B.bssn_tile_name(tile),
           "stage_launch_ms": stage_ms / max(stage_n, 1), "stage_launches": stage_n,
           "boundary_launch_ms": bc_ms / max(bc_n, 1), "boundary_launches": bc_n, "clocks": clk}
    if e2e:
        # two read-back buffers: the copy of step n's state to the host runs
        # on the library's copy stream while step n+1's state is uploaded
        host_in = torch.empty(evo.shape, dtype=torch.float64, pin_memory=True).numpy()
        host_out = [torch.empty(evo.shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        host_in[...], _ = evo.get_state()
        evo.enable_copy_staging()  # the copies overlap the steps as well as each other
        e2e_steps = max(2, steps)
        barrier(world)
        t0 = time.perf_counter()
        for s_ in range(e2e_steps):
            B.bssn_set_state_async(evo.ctx, host_in, 0.0)
            evo.rk4_step(1)
            B.bssn_get_state_async(evo.ctx, host_out[s_ % 2])
        B.bssn_wait_state(evo.ctx)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        out["e2e"] = {"value": pts * e2e_steps * world / e2e_s / 1e6, "unit": "Mpoint-updates/s",
                      "h2d_bytes_per_step": host_in.nbytes, "d2h_bytes_per_step": host_in.nbytes,
                      "steps": e2e_steps,
                      "copies": "pinned; device staging areas: the upload of step n+1 and the read-back "
                                "of step n overlap each other and the steps"}
    evo.close()
    del evo
    torch.cuda.empty_cache()
    return out


def hbm_roofline(run, precision, kernel, traffic_per_point):
    """The dominant (stage) kernel against HBM: algorithmic bytes of one stage
    launch (a quarter of the per-step bytes, per interior point) over its
    mean launch duration."""
    pts = N_SIDE ** 3
    bytes_launch = ALG_BYTES_PER_POINT_STEP[precision] / 4.0 * pts
    gbs = bytes_launch / (run["stage_launch_ms"] * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": gbs, "peak": HBM_MEASURED_GBS, "unit": "GB/s",
            "frac": gbs / HBM_MEASURED_GBS,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)",
            "algorithmic_bytes_per_launch": bytes_launch,
            "traffic": traffic_per_point * pts if traffic_per_point and N_SIDE == TRAFFIC_N else None,
            "launch_ms": run["stage_launch_ms"], "launches": run["stage_launches"],
            "boundary_launch_ms": run["boundary_launch_ms"]}


def run_ours(args):
    import torch

    from paper_1111_3344_gb300 import bssn as B
    rank, world, local = dist_setup(args.gpus)
    run = puncture_run(args, args.precision, world, local, args.steps)
    pts = N_SIDE ** 3
    mixed = args.precision == "mixed"
    rows = run["tile"] in ROWS_TILES and N_SIDE % 32 == 0
    if mixed:
        kernel = "stage_mixed_tma_kernel" if run["tile"].startswith("tma") else "stage_mixed_kernel"
        roofline = hbm_roofline(run, "mixed", kernel, STAGE_TRAFFIC_PER_POINT.get(("mixed", run["tile"])))
    elif args.precision == "ff":
        roofline = hbm_roofline(run, "ff", "stage_ff_kernel", None)
    else:
        kernel = "stage_fp64_blocks_kernel" if rows else "stage_fp64_kernel"
        roofline = hbm_roofline(run, "fp64", kernel, STAGE_TRAFFIC_PER_POINT.get(("fp64", run["tile"])))
        peaks = measured_peaks(B, torch, torch.cuda.Stream())
        flop_pt = FLOP_PER_POINT_RHS_ROWS if rows else FLOP_PER_POINT_RHS
        dpinst_pt = DPINST_PER_POINT_RHS_ROWS if rows else DPINST_PER_POINT_RHS
        sec = run["stage_launch_ms"] * 1e-3
        # the pipe that binds the float64 stage: executed float64 work of a
        # launch over the float64 FMA rate measured in this run
        roofline["binding"] = {
            "bound": "alu", "pipe": "fp64", "unit": "GFLOP/s",
            "achieved": flop_pt * pts / sec / 1e9, "peak": peaks["fp64_gflops"],
            "frac": flop_pt * pts / sec / 1e9 / peaks["fp64_gflops"],
            "peak_source": "measured in this run (bssn_peak_probe, float64 FMA chains)",
            "executed_flop_per_point": flop_pt,
            "fp64_issue_frac": dpinst_pt * pts / sec / (peaks["fp64_gflops"] * 1e9 / 2),
            "oracle_flop_per_point_rhs": ORACLE_FLOP_PER_POINT_RHS,
            "nominal_fp64_gflops": FP64_NOMINAL_GFLOPS}
        roofline["measured_peaks"] = peaks
    line = {
        "metric": {"mixed": "BSSN RK4 point-updates/s (mixed FP32 RHS / FP64 state, Brill-Lindquist puncture 128^3)",
                   "ff": "BSSN RK4 point-updates/s (double-word FP32 RHS / FP64 state, Brill-Lindquist puncture "
                         "128^3)"}.get(args.precision,
                                       "BSSN RK4 point-updates/s (FP64, Brill-Lindquist puncture 128^3)"),
        "value": run["value"], "unit": "Mpoint-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": run["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "ff": "f32x2+f64"}.get(args.precision, "f64"),
        "data": "synthetic",
        "config": {"workload": "single Brill-Lindquist puncture M=1, 128^3 on [-8,8]^3, W, 1+log, "
                               "Gamma-driver eta=2, Sommerfeld, RK4 dt=0.25h",
                   "global_batch": world, "grid": [N_SIDE] * 3, "parallelism": f"replicas{world}",
                   "precision": args.precision, "tile": run["tile"],
                   "l2": "inputs larger than L2 (4 float64 registers of 469 MB each)"},
        "roofline": roofline,
        "rhs_evaluations_per_s": 4.0 * run["value"] * 1e6,  # four right-hand sides per point-update
        "e2e": run["e2e"],
        # the split mixed stage is two kernels per stage (stencils, algebra);
        # a float64 boundary pass is two (anchor pass, ghost points)
        "gpu_launches": run["stage_launches"] * (2 if run["tile"].startswith("split") else 1)
                        + run["boundary_launches"] * (2 if args.precision == "fp64" else 1),
        "clocks": run["clocks"],
    }
    if world == 1 and not args.no_extras and args.precision == "fp64":
        line.update(extras(args))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def extras(args):
    """The rest of the benchmark's metric, each part with its own CUDA-event
    timing and clock sample: the mixed-precision puncture at 128^3, the
    batched 64-binary workload in both precisions, and a labelled sample of
    the served workload whose arrival rate is 0.8x a capacity measured on the
    served request mix in this run."""
    import torch
    mixed = puncture_run(args, "mixed", 1, 0, args.steps)
    kernel = "stage_mixed_tma_kernel" if mixed["tile"].startswith("tma") else "stage_mixed_kernel"
    out = {"mixed": {
        "metric": "BSSN RK4 point-updates/s (mixed FP32 RHS / FP64 state, Brill-Lindquist puncture 128^3)",
        "value": mixed["value"], "unit": "Mpoint-updates/s", "ms_per_step": mixed["ms"] / mixed["steps"],
        "steps": mixed["steps"], "dtype": "f32+f64", "tile": mixed["tile"],
        "roofline": hbm_roofline(mixed, "mixed", kernel, STAGE_TRAFFIC_PER_POINT.get(("mixed", mixed["tile"]))),
        "e2e": mixed["e2e"], "gpu_launches": mixed["stage_launches"] + mixed["boundary_launches"],
        "clocks": mixed["clocks"]}}
    bsteps = max(2, args.steps // 4)
    out["batched"] = {prec: batched_run(args, prec, steps=bsteps) for prec in ("fp64", "mixed", "ff")}
    torch.cuda.empty_cache()
    out["served_sample"] = served_run(args, "mixed", requests=args.served_sample)
    return out


def _bl_params(member, precision):
    from paper_1111_3344_gb300.bssn import Params
    h = member["h"]
    return Params(n=member["n"], xmin=member["xmin"], h=h, boundary="sommerfeld", conformal="W",
                  slicing="1+log", shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * h,
                  precision=precision, w_fp64_threshold=0.2, r_excise=1.0)


def _make_batch(B, params_list, precision):
    need = sum(B.Batch.member_bytes(p) for p in params_list) + (64 << 20)
    return B.Batch(precision, pool_bytes=need, max_members=max(len(params_list), 1))


def batched_run(args, precision, steps=None, members=None):
    """64 time-symmetric Brill-Lindquist binaries (masses U[0.3,0.7], separations
    U[2,6], grids from {48,64,96,128}^3, seed 1111) advanced together, one
    launch per RK4 stage (plus one boundary launch) under a CUDA graph; steps
    timed with CUDA events on the batch's stream."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    from paper_1111_3344_gb300 import inputs
    torch.cuda.set_device(0)
    steps = args.steps if steps is None else steps
    mems = inputs.binary_bl_batch(seed=1111, count=members or args.members)
    params = [_bl_params(m, precision) for m in mems]
    batch = _make_batch(B, params, precision)
    for m, p in zip(mems, params):
        mid = batch.add(p)
        bl = [len(m["punctures"])] + [v for q in m["punctures"] for v in q]
        batch.set_initial_data(mid, "bl", bl)
    best, tile_ms = batch.autotune(reps=2)
    step_ms = {}
    if args.tile and args.tile in tile_ms:
        best = list(tile_ms).index(args.tile)
        batch.set_tile(best)
    else:
        best, step_ms = confirm_by_steps(tile_ms, batch.set_tile, batch.step, batch.stream)
    batch.step(args.warmup)
    batch.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(batch.stream)
    batch.step(steps)
    stop.record(batch.stream)
    stop.synchronize()
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    pts = sum(p.n[0] * p.n[1] * p.n[2] for p in params)
    # launches per step: a stage and a boundary launch per RK4 stage; the
    # one-block-per-tile float64 configurations launch the members with full
    # tiles and the others separately
    tname = list(tile_ms)[best]
    stage_launches, bc_launches = 1, 1
    if tname.startswith(("tiles", "fftiles")) and precision in ("fp64", "ff"):
        tx, ty, tz = (int(v) for v in tname.split("tiles")[1].split("/")[0].split("x"))
        full = [tx == 32 and p.n[0] % 32 == 0 and p.n[1] % ty == 0 and p.n[2] % tz == 0 for p in params]
        stage_launches = int(any(full)) + int(not all(full))
    elif tname.startswith("members"):
        # per member and stage: its stage kernel and its Sommerfeld boundary
        # (float64: the anchor pass and the ghost-point pass)
        stage_launches = len(params)
        bc_launches = len(params) * (2 if precision == "fp64" else 1)
    batch.close()
    del batch
    torch.cuda.empty_cache()
    return {"metric": f"batched BSSN RK4 point-updates/s ({precision})",
            "value": pts * steps / (ms * 1e-3) / 1e6, "unit": "Mpoint-updates/s", "steps": steps,
            "ms_per_step": ms / steps, "dtype": {"fp64": "f64", "mixed": "f32+f64", "ff": "f32x2+f64"}[precision],
            "workload": f"{len(params)} Brill-Lindquist binaries, grids {{48,64,96,128}}^3, seed 1111, "
                        f"{steps} of the configuration's 100 steps",
            "interior_points": pts, "tile": tname,
            "autotune_ms_per_stage": {k: round(v, 3) for k, v in tile_ms.items() if v >= 0},
            "confirm_ms_per_step": {k: round(v, 3) for k, v in step_ms.items()},
            "launches_per_step": 4 * (stage_launches + bc_launches),
            "gpu_launches": 4 * (stage_launches + bc_launches) * steps,
            "graph": True, "clocks": clk}


def served_requests(count, precision, seed=3344):
    """The served workload's request stream: grids from {32,...,192}^3, 50 to
    400 steps, Brill-Lindquist binaries as in the batched workload (punctures
    snapped half a cell off the grid)."""
    rng = np.random.default_rng(seed)
    sizes = [32, 48, 64, 96, 128, 160, 192]
    reqs = []
    for _ in range(count):
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
        reqs.append((_bl_params(mem, precision), [2, m1, x1, 0.0, 0.0, m2, x2, 0.0, 0.0], steps))
    return rng, reqs


def served_capacity(reqs, precision, steps=3):
    """Capacity of the serving path on its own request mix, M point-updates/s:
    the first requests of the stream (up to 24) resident together in one batch
    with the serving path's kernels (the default configuration of a new batch,
    which the server runs), `steps` RK4 steps timed with CUDA events."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    sample = reqs[:24]
    params = [p for p, _, _ in sample]
    batch = _make_batch(B, params, precision)
    for p, idp, _ in sample:
        batch.set_initial_data(batch.add(p), "bl", idp)
    batch.step(1)
    batch.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(batch.stream)
    batch.step(steps)
    e1.record(batch.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    batch.close()
    del batch
    torch.cuda.empty_cache()
    pts = sum(p.n[0] * p.n[1] * p.n[2] for p in params)
    return pts * steps / (ms * 1e-3) / 1e6, len(sample)


def served_run(args, precision, requests, keep_norms=False):
    """Poisson arrivals of puncture evolutions admitted by HBM budget into a
    continuous-batching server: the arrival rate is 0.8x the capacity
    measured on the same request mix just before; reports p50/p99 time from
    submission to completion, the queueing part of them, and throughput both
    over wall-clock time and over the time the server spent stepping."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    torch.cuda.set_device(0)
    rng, reqs = served_requests(requests, precision)
    capacity, cap_n = served_capacity(reqs, precision)
    work = sum(p.n[0] ** 3 * st for p, _, st in reqs)
    lam = 0.8 * capacity * 1e6 / (work / len(reqs))
    gaps = rng.exponential(1.0 / lam, size=len(reqs))
    budget = int(args.budget_gb * (1 << 30))
    srv = B.Server(precision, budget_bytes=budget)
    srv.set_policy(args.serve_policy, args.serve_min_points)
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    tickets = []
    for (p, idp, st), gap in zip(reqs, gaps):
        time.sleep(gap)
        tickets.append(srv.submit(p, "bl", idp, st))
    lats, queued, fails, all_norms = [], [], 0, []
    for t in tickets:
        st, norms, lat = srv.wait(t, timeout=3600)
        lats.append(lat)
        queued.append(srv.detail(t)[1])
        fails += st != 0
        all_norms.append(norms)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    stats = srv.stats()
    srv.close()
    lats, queued = np.array(lats), np.array(queued)
    p99 = float(np.percentile(lats, 99))
    i99 = int(np.argmin(np.abs(lats - p99)))
    extra = {"norms": np.array(all_norms)} if keep_norms else {}
    return {**extra, "metric": "served BSSN evolutions: p50/p99 completion latency, aggregate point-updates/s",
            "value": stats["point_updates"] / wall / 1e6, "unit": "Mpoint-updates/s",
            "busy_value": stats["point_updates"] / stats["busy_s"] / 1e6,
            "p50_s": float(np.percentile(lats, 50)), "p99_s": p99,
            "p99_queued_s": float(queued[i99]), "mean_queued_s": float(queued.mean()),
            "failed": int(fails), "wall_s": wall, "busy_s": stats["busy_s"],
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "ff": "f32x2+f64"}[precision],
            "workload": f"first {len(reqs)} requests of the served stream (seed 3344): Poisson arrivals of "
                        f"Brill-Lindquist binaries, grids 32^3..192^3, 50..400 steps",
            "policy": args.serve_policy,
            "min_points": args.serve_min_points if args.serve_policy == "shortest" else None,
            "lambda_per_s": lam, "capacity_mpts": capacity,
            "capacity_source": f"{cap_n} requests of the same stream resident in one batch, 3 steps timed "
                               "with CUDA events in this run; lambda = 0.8 x capacity / mean work per request",
            "budget_gb": args.budget_gb, "point_updates": work, "clocks": clk}


def run_batched(args):
    line = batched_run(args, args.precision)
    line.update({"n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "data": "synthetic"})
    print(json.dumps(line))


def run_served(args):
    line = served_run(args, args.precision, args.requests)
    line.update({"n_gpus": 1, "higher_is_better": True, "data": "synthetic"})
    print(json.dumps(line))


def run_precision_served(args):
    """The served workload's first args.requests requests through the server
    in float64 and in each of args.variants (mixed, ff), each at 0.8x its own
    measured capacity (the same seeded arrival gaps scaled by its rate): every
    request's 16 constraint norms against the same request's float64 norms,
    and the serving throughput (point-updates over the seconds the server
    spent stepping, and over wall time) against float64."""
    variants = [v for v in args.variants.split(",") if v in ("mixed", "ff")]
    runs = {prec: served_run(args, prec, args.requests, keep_norms=True) for prec in ["fp64"] + variants}
    ref = runs["fp64"]["norms"]
    res = {}
    for prec in variants:
        r = runs[prec]
        rel = np.abs(r["norms"] - ref) / np.where(ref != 0, np.abs(ref), np.inf)
        res[prec] = {"busy_Mpts": r["busy_value"], "wall_Mpts": r["value"],
                     "busy_speedup_over_fp64": r["busy_value"] / runs["fp64"]["busy_value"],
                     "p50_s": r["p50_s"], "p99_s": r["p99_s"], "failed": r["failed"],
                     "max_constraint_norm_rel_diff": float(rel.max()),
                     "max_rel_diff_full_domain": float(rel[:, :8].max()),
                     "max_rel_diff_excised": float(rel[:, 8:].max()),
                     "requests_within_1e-6": int((rel.max(axis=1) <= 1e-6).sum()),
                     "clocks": r["clocks"]}
    f = runs["fp64"]
    line = {"metric": "served reduced-precision forms vs float64: per-request constraint-norm relative "
                      "difference, serving throughput",
            "workload": f"first {args.requests} requests of the served stream (seed 3344), each form at 0.8x "
                        f"its own measured capacity, policy {args.serve_policy}",
            "requests": args.requests, "bar": "constraint norms within 1e-6 relative of the float64 run",
            "fp64": {"busy_Mpts": f["busy_value"], "wall_Mpts": f["value"], "p50_s": f["p50_s"],
                     "p99_s": f["p99_s"], "failed": f["failed"], "clocks": f["clocks"]},
            "variants": res, "n_gpus": 1, "data": "synthetic"}
    print(json.dumps(line))


def run_precision(args):
    """Reduced-precision forms against float64 on the same GPU: the puncture at
    args.n^3 (the configuration is 256^3, 100 steps) evolved args.steps RK4
    steps in float64 and in each of args.variants; for each variant the
    per-field L2 and Linf of the state difference from the float64 run
    (interior points; absolute and relative to the field's largest float64
    value), the relative difference of every constraint norm (full domain and
    excised), the time of the steps (CUDA events) and the speedup."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    torch.cuda.set_device(0)
    variants = [v for v in args.variants.split(",") if v and v != "fp64"]
    out = {}
    for prec in ["fp64"] + variants:
        evo = B.Evolution(workload_params(prec))
        evo.set_initial_data("bl", BL_P)
        _, tile_ms = B.bssn_autotune(evo.ctx, reps=2)
        tile, _ = confirm_by_steps(tile_ms, lambda c: B.bssn_set_tile(evo.ctx, c), evo.rk4_step, evo.stream)
        evo.set_initial_data("bl", BL_P)  # the timed run starts at t = 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(evo.stream)
        evo.rk4_step(args.steps)
        e1.record(evo.stream)
        e1.synchronize()
        st, _ = evo.get_state()
        out[prec] = (st, evo.constraints(), e0.elapsed_time(e1) * 1e-3, B.bssn_tile_name(tile))
        evo.close()
        del evo
        torch.cuda.empty_cache()
    s64, c64, t64, tile64 = out["fp64"]
    g = 3
    names = ["chi", "gt_xx", "gt_xy", "gt_xz", "gt_yy", "gt_yz", "gt_zz", "trK", "At_xx", "At_xy",
             "At_xz", "At_yy", "At_yz", "At_zz", "Gt_x", "Gt_y", "Gt_z", "alpha", "beta_x", "beta_y",
             "beta_z", "B_x", "B_y", "B_z"]
    ref = np.abs(s64[:, g:-g, g:-g, g:-g]).reshape(24, -1).max(axis=1)
    cn = ["H", "Mx", "My", "Mz"]
    keys = [f"{k}_{n}_{s}" for s in ("full", "excised") for k in ("L2", "Linf") for n in cn]
    res = {}
    for prec in variants:
        sv, cv, tv, tilev = out[prec]
        d = (sv - s64)[:, g:-g, g:-g, g:-g].reshape(24, -1)
        l2 = np.sqrt((d ** 2).mean(axis=1))
        linf = np.abs(d).max(axis=1)
        fields = {nm: {"L2": float(l2[f]), "Linf": float(linf[f]), "L2_rel": float(l2[f] / max(ref[f], 1e-300)),
                       "Linf_rel": float(linf[f] / max(ref[f], 1e-300)), "max_abs_fp64": float(ref[f])}
                  for f, nm in enumerate(names)}
        rel = {k: float(abs(a - b) / abs(b)) if b != 0 else None for k, a, b in zip(keys, cv, c64)}
        res[prec] = {"seconds": tv, "speedup_over_fp64": t64 / tv, "tile": tilev,
                     "max_constraint_norm_rel_diff": max(v for v in rel.values() if v is not None),
                     "constraint_norm_rel_diff": rel, "constraint_norms": dict(zip(keys, cv.tolist())),
                     "max_field_Linf_rel": float(max(f["Linf_rel"] for f in fields.values())),
                     "fields": fields}
    line = {"metric": "reduced-precision forms vs float64: per-field state error and constraint-norm relative "
                      "difference, speedup",
            "workload": f"single Brill-Lindquist puncture M=1, {args.n}^3 on [-8,8]^3, {args.steps} RK4 steps",
            "grid": args.n, "steps": args.steps, "bar": "constraint norms within 1e-6 relative of the float64 run",
            "fp64": {"seconds": t64, "tile": tile64, "constraint_norms": dict(zip(keys, c64.tolist()))},
            "variants": res}
    print(json.dumps(line))


def run_precision_batched(args):
    """The batched workload (64 Brill-Lindquist binaries, seed 1111) advanced
    args.steps RK4 steps (the configuration's 100) in float64 and in each of
    args.variants (mixed, ff); for each variant, every member's 16 constraint
    norms against the same member's float64 norms, the largest relative
    difference over members (and over the full-domain and the excised norms
    separately), and the time of the steps (CUDA events) against float64."""
    import torch

    from paper_1111_3344_gb300 import bssn as B
    from paper_1111_3344_gb300 import inputs
    torch.cuda.set_device(0)
    mems = inputs.binary_bl_batch(seed=1111, count=args.members)
    variants = [v for v in args.variants.split(",") if v in ("mixed", "ff")]
    norms, secs, tiles = {}, {}, {}
    for prec in ["fp64"] + variants:
        params = [_bl_params(m, prec) for m in mems]
        batch = _make_batch(B, params, prec)
        ids = []
        for m, p in zip(mems, params):
            mid = batch.add(p)
            batch.set_initial_data(mid, "bl", [len(m["punctures"])] + [v for q in m["punctures"] for v in q])
            ids.append(mid)
        best, tile_ms = batch.autotune(reps=1)
        best, _ = confirm_by_steps(tile_ms, batch.set_tile, batch.step, batch.stream)
        # start the timed run from t = 0
        for mid, m in zip(ids, mems):
            batch.set_initial_data(mid, "bl", [len(m["punctures"])] + [v for q in m["punctures"] for v in q])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(batch.stream)
        batch.step(args.steps)
        e1.record(batch.stream)
        e1.synchronize()
        secs[prec] = e0.elapsed_time(e1) * 1e-3
        tiles[prec] = list(tile_ms)[best]
        norms[prec] = np.array([batch.constraints(mid) for mid in ids])
        batch.close()
        del batch
        torch.cuda.empty_cache()
    ref = norms["fp64"]
    res = {}
    for prec in variants:
        rel = np.abs(norms[prec] - ref) / np.where(ref != 0, np.abs(ref), np.inf)
        res[prec] = {"seconds": secs[prec], "speedup_over_fp64": secs["fp64"] / secs[prec], "tile": tiles[prec],
                     "max_constraint_norm_rel_diff": float(rel.max()),
                     "max_rel_diff_full_domain": float(rel[:, :8].max()),
                     "max_rel_diff_excised": float(rel[:, 8:].max()),
                     "median_over_members_of_max": float(np.median(rel.max(axis=1))),
                     "members_within_1e-6": int((rel.max(axis=1) <= 1e-6).sum())}
    pts = sum(m["n"][0] * m["n"][1] * m["n"][2] for m in mems)
    line = {"metric": "batched reduced-precision forms vs float64: per-member constraint-norm relative difference, "
                      "speedup",
            "workload": f"{len(mems)} Brill-Lindquist binaries, grids {{48,64,96,128}}^3, seed 1111, "
                        f"{args.steps} RK4 steps each",
            "members": len(mems), "steps": args.steps, "interior_points": pts,
            "bar": "constraint norms within 1e-6 relative of the float64 run",
            "fp64": {"seconds": secs["fp64"], "tile": tiles["fp64"],
                     "Mpoint_updates_per_s": pts * args.steps / secs["fp64"] / 1e6},
            "variants": res}
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
    peaks = measured_peaks(B, torch, stream)
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
                     "peak": peaks["fp64_gflops"], "unit": "GFLOP/s (FP64)",
                     "peak_source": "measured in this run (bssn_peak_probe, float64 FMA chains)",
                     "frac": top["fp64_gflops"] / peaks["fp64_gflops"], "traffic": None},
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
    ap.add_argument("--precision", choices=["fp64", "mixed", "ff"], default=None,
                    help="default: mixed for the served workload (its configuration), float64 otherwise")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["puncture", "batched", "served", "precision", "precision_batched",
                                           "precision_served",
                                           "analysis"],
                    default="puncture",
                    help="puncture: the benchmark line (single 128^3 puncture); batched / served: "
                         "the multi-evolution workloads, reported on their own lines")
    ap.add_argument("--tile", default=None, help="stage-kernel configuration name (default: autotune)")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="puncture workload: print the float64 line only, without the mixed, batched and "
                         "served parts of the metric")
    ap.add_argument("--serve-policy", choices=["all", "shortest"], default="shortest",
                    help="server: step every resident request, or the shortest remaining work first")
    ap.add_argument("--serve-min-points", type=float, default=float(1 << 21),
                    help="shortest-first policy: interior points a step advances at least")
    ap.add_argument("--served-sample", type=int, default=32,
                    help="requests of the served stream in the default line's served sample")
    ap.add_argument("--variants", default="mixed,mixed_ks64,ff",
                    help="precision workload: the forms compared with float64 (mixed, mixed_ks64, ff)")
    ap.add_argument("--n", type=int, default=128,
                    help="grid points per side (128 is the benchmark workload; smaller sizes are "
                         "for profiling captures only)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "mixed" if args.workload == "served" else "fp64"
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
    elif args.workload == "precision_batched":
        run_precision_batched(args)
    elif args.workload == "precision_served":
        run_precision_served(args)
    elif args.workload == "analysis":
        run_analysis(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
