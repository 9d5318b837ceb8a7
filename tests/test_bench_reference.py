"""The benchmark's reference arm (`bench.py --impl reference`) runs on the host:
it times the CPU oracle on a bounded sample of the benchmark workload and
prints one JSON line with the keys the benchmark contract names, on the same
metric as the GPU line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "BSSN RK4 point-updates/s (FP64, Brill-Lindquist puncture 128^3)"
    assert d["unit"] == "Mpoint-updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_bench_oracle_flop_count_is_the_oracles():
    """The operation count bench.py reports beside the roofline is the one the
    instrumented oracle counts for the benchmark configuration (W variant,
    1+log slicing, Gamma-driver shift, Sommerfeld grid) at an interior point."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    n = 12
    cfg = O.Config(n=(n,) * 3, xmin=(-1.5,) * 3, h=0.25, periodic=False, use_w=True, slicing="1+log",
                   shift="gamma-driver", eta=2.0, punctures=[(1.0, 0.0, 0.0, 0.0)])
    st = O.initial_data(cfg, "bl", [1, 1.0, 0.0, 0.0, 0.0])
    c = O.rhs_opcount(cfg, st, (9, 8, 7))
    assert c["add"] + c["mul"] + c["div"] == bench.ORACLE_FLOP_PER_POINT_RHS


def test_hbm_roofline_arithmetic():
    """The roofline object of the bench line: achieved = algorithmic bytes of
    one stage launch (a quarter of the per-step bytes per interior point, times
    the interior points) over the mean launch time; frac = achieved over the
    measured copy bandwidth; traffic = the captured DRAM bytes per point times
    the points, only at the grid size the capture was made at."""
    sys.path.insert(0, ROOT)
    import bench
    run = {"stage_launch_ms": 7.25, "stage_launches": 80, "boundary_launch_ms": 0.3}
    n_saved = bench.N_SIDE
    try:
        bench.N_SIDE = 128
        r = bench.hbm_roofline(run, "fp64", "stage_fp64_blocks_kernel", 937.2)
        pts = 128 ** 3
        assert r["algorithmic_bytes_per_launch"] == 3072.0 / 4.0 * pts
        assert abs(r["achieved"] - 768.0 * pts / 7.25e-3 / 1e9) < 1e-9
        assert abs(r["frac"] - r["achieved"] / bench.HBM_MEASURED_GBS) < 1e-15
        assert r["traffic"] == 937.2 * pts and r["unit"] == "GB/s" and r["bound"] == "hbm"
        r = bench.hbm_roofline(run, "mixed", "stage_mixed_tma_kernel", None)
        assert r["algorithmic_bytes_per_launch"] == 2496.0 / 4.0 * pts and r["traffic"] is None
        bench.N_SIDE = 64  # not the capture size: no traffic figure
        r = bench.hbm_roofline(run, "fp64", "stage_fp64_blocks_kernel", 937.2)
        assert r["traffic"] is None and r["algorithmic_bytes_per_launch"] == 768.0 * 64 ** 3
    finally:
        bench.N_SIDE = n_saved
