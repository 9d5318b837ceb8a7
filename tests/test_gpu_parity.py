"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar (float64 path): per field, normwise relative error <= 1e-12 per
right-hand-side call, or, where the oracle's magnitude of the terms at a point
exceeds the field's scale (a small difference of far larger terms), 1e-12 of
that magnitude (cases.rounding_aware_errors); RK4 steps compound a few calls,
so their bar is 1e-11.  Inputs come from the oracle or from the seeded generators in
paper_1111_3344_gb300/inputs.py, never from the CUDA path."""
import math

import numpy as np
import pytest

import oracle as O
from cases import bl_params, gpu_params, normwise_errors, oracle_cfg, rounding_aware_errors
from paper_1111_3344_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-12
TOL_STEP = 1e-11


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


def _evo(case):
    from paper_1111_3344_gb300.bssn import Evolution
    return Evolution(gpu_params(case))


BL1 = dict(n=(37, 21, 19), xmin=(-4.1, -2.3, -2.2), h=0.2203, boundary="sommerfeld",
           punctures=[(1.0, 0.05, -0.02, 0.01)], r_excise=0.8)
CASES = {
    # moving-puncture setting with a perturbed state exercising every term; ragged tiles
    "bl_w_1pluslog_sommerfeld": dict(BL1, conformal="W", slicing="1+log", shift="gamma-driver",
                                     eta=2.0, q_R=1.7),
    "bl_phi_harmonic_sommerfeld": dict(BL1, conformal="phi", slicing="harmonic", shift="gamma-driver",
                                       eta=0.5),
    "random_periodic_w_geodesic": dict(n=(33, 9, 12), xmin=(-0.5, -0.2, -0.3), h=1.0 / 33,
                                       boundary="periodic", conformal="W", slicing="geodesic"),
    "random_periodic_phi_frozen": dict(n=(16, 40, 8), xmin=(0.0, 0.0, 0.0), h=0.05,
                                       boundary="periodic", conformal="phi", slicing="1+log",
                                       shift="frozen"),
    "minimal_grid": dict(n=(4, 4, 4), xmin=(-0.2, -0.2, -0.2), h=0.1, boundary="sommerfeld",
                         conformal="W"),
}


def _state_for(name, case):
    cfg = oracle_cfg(case)
    if case.get("punctures"):
        bg = O.initial_data(cfg, "bl", bl_params(case))
        return inputs.random_state(7, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    return inputs.random_state(11, case["n"], case["xmin"], case["h"], amp=0.1)


@pytest.mark.parametrize("kind", ["flat", "gauge_wave", "bl", "kasner"])
@pytest.mark.parametrize("conformal", ["W", "phi"])
def test_initial_data_parity(torch_cuda, kind, conformal):
    case = dict(n=(20, 13, 9), xmin=(-0.5, -0.7, -0.3), h=0.07, boundary="sommerfeld",
                conformal=conformal, punctures=[(0.7, 0.05, 0.0, 0.0), (0.4, -0.3, 0.1, 0.0)])
    p = {"flat": [], "gauge_wave": [0.01, 1.0], "bl": bl_params(case), "kasner": [1.3]}[kind]
    evo = _evo(case)
    evo.set_initial_data(kind, p)
    got, t = evo.get_state()
    want = O.initial_data(oracle_cfg(case), kind, p)
    e = normwise_errors(got, want)
    assert e.max() <= 1e-13, e
    assert t == 0.0


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_parity(torch_cuda, name):
    case = CASES[name]
    st = _state_for(name, case)
    evo = _evo(case)
    reg = evo.numpy_to_register(st)
    got = evo.register_to_numpy(evo.rhs(reg))
    want = O.rhs(oracle_cfg(case), st)
    e = normwise_errors(got, want)
    assert e.max() <= TOL_RHS, dict(zip(O.FIELD_NAMES, e))
    # every field's right-hand side is non-trivial in the perturbed cases
    if name.startswith(("bl_", "random_periodic_w")):
        assert (np.abs(want).reshape(24, -1).max(axis=1)[:18] > 0).all()


@pytest.mark.parametrize("name", ["bl_w_1pluslog_sommerfeld", "random_periodic_w_geodesic",
                                  "random_periodic_phi_frozen", "minimal_grid"])
def test_rk4_parity(torch_cuda, name):
    case = CASES[name]
    st = _state_for(name, case)
    evo = _evo(case)
    evo.set_state(st, 0.0)
    evo.rk4_step(3)
    got, t = evo.get_state()
    want = O.rk4(oracle_cfg(case), st, 3)
    e = normwise_errors(got, want)
    assert e.max() <= TOL_STEP, dict(zip(O.FIELD_NAMES, e))
    assert t == pytest.approx(3 * case.get("dt", 0.25 * case["h"]))


def test_zero_steps_leave_state_unchanged(torch_cuda):
    case = CASES["bl_w_1pluslog_sommerfeld"]
    st = _state_for("bl", case)
    evo = _evo(case)
    evo.set_state(st, 1.5)
    evo.rk4_step(0)
    got, t = evo.get_state()
    assert np.array_equal(got, st) and t == 1.5


@pytest.mark.parametrize("name", ["bl_w_1pluslog_sommerfeld", "bl_phi_harmonic_sommerfeld",
                                  "random_periodic_w_geodesic"])
def test_constraint_norm_parity(torch_cuda, name):
    case = CASES[name]
    st = _state_for(name, case)
    evo = _evo(case)
    evo.set_state(st, 0.0)
    if case.get("punctures"):
        evo.set_initial_data("bl", bl_params(case))  # registers the punctures for excision
        evo.set_state(st, 0.0)
    got = evo.constraints()
    want, _, _ = O.constraints(oracle_cfg(case), st)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def test_flat_space_stays_flat_on_gpu(torch_cuda):
    case = dict(n=(12, 12, 12), xmin=(-0.5,) * 3, h=1 / 12, boundary="sommerfeld", conformal="W")
    evo = _evo(case)
    evo.set_initial_data("flat")
    st0, _ = evo.get_state()
    evo.rk4_step(5)
    st, _ = evo.get_state()
    assert np.array_equal(st, st0)
    assert np.all(evo.constraints() == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tile_configs_agree_and_are_deterministic(torch_cuda, precision):
    """Every stage-kernel tile configuration evaluates the same per-point
    formulas; ptxas may fuse multiply-adds differently under different register
    budgets, so configurations agree to rounding (not bit for bit), while each
    configuration is bit-reproducible.  The autotuner only picks among them."""
    from paper_1111_3344_gb300 import bssn as B
    case = dict(CASES["bl_w_1pluslog_sommerfeld"], precision=precision, w_fp64_threshold=0.3)
    st = _state_for("bl", case)
    runs = {}
    for cfg in range(B.bssn_tile_count()):
        name = B.bssn_tile_name(cfg)
        mixed_only = name.startswith(("tma", "split")) or name in ("32x4x1/4", "32x4x1/6")
        if (precision == "fp64" and mixed_only) or name.startswith("ff"):
            evo = _evo(case)
            # the TMA-staged, split and register-capped mixed kernels are mixed-only, the
            # ff kernels double-word only
            with pytest.raises(B.BssnError):
                B.bssn_set_tile(evo.ctx, cfg)
            evo.close()
            continue
        outs = []
        for _ in range(2):
            evo = _evo(case)
            B.bssn_set_tile(evo.ctx, cfg)
            evo.set_state(st, 0.0)
            evo.rk4_step(2)
            outs.append(evo.get_state()[0])
            evo.close()
        assert np.array_equal(outs[0], outs[1]), B.bssn_tile_name(cfg)
        runs[cfg] = outs[0]
    tol = 1e-13 if precision == "fp64" else 1e-4
    for cfg, got in runs.items():
        e = normwise_errors(got, runs[0])
        assert e.max() <= tol, (B.bssn_tile_name(cfg), e.max())
    evo = _evo(case)
    evo.set_state(st, 0.0)
    best, times = B.bssn_autotune(evo.ctx, reps=2)
    assert 0 <= best < B.bssn_tile_count() and len(times) == B.bssn_tile_count()
    assert min(times.values()) == times[B.bssn_tile_name(best)]
    assert best in runs
    evo.rk4_step(2)
    assert np.array_equal(evo.get_state()[0], runs[best])


@pytest.mark.parametrize("name,box,periodic", [("ks_wavy", (1.5, 2.5), False), ("flat_wavy", (-0.5, 0.5), False),
                                               ("gauge_wave", (-0.5, 0.5), True)])
@pytest.mark.parametrize("conformal", ["W", "phi"])
def test_set_adm_parity(torch_cuda, name, box, periodic, conformal):
    """General ADM -> BSSN (Gt by differences, cubic extrapolation on the outer
    layers) against the oracle, on exact-spacetime ADM data."""
    import exact_solutions as E
    lo, hi = box
    n = (20, 17, 23)
    case = dict(n=n, xmin=(lo, lo, lo), h=(hi - lo) / 20, boundary="periodic" if periodic else "sommerfeld",
                conformal=conformal)
    cfg = oracle_cfg(case)
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    _, _, grad = E.evaluate(name, Xc, Yc, Zc, use_w=conformal == "W")
    adm = np.ascontiguousarray(grad["adm"])
    want = O.adm_to_bssn_fd(cfg, adm)
    evo = _evo(case)
    evo.set_adm(adm, 0.25)
    got, t = evo.get_state()
    # interior points: normwise per field within 1e-12
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    e = normwise_errors(got[inner], want[inner])
    assert e.max() <= 1e-12, dict(zip(O.FIELD_NAMES, e))
    # ghost layers: the cubic extrapolation v = 4 v1 - 6 v2 + 4 v3 - v4 carries
    # an input error forward with gain |4|+|6|+|4|+|1| = 15 on the first layer,
    # 4*15 + 11 = 71 on the second and 4*71 + 6*15 + 5 = 379 on the third, so
    # the ghosts agree to 379 times the interior error plus the rounding of the
    # sums themselves (a few ulp of the field's scale per layer).
    d_in = np.abs(got[inner] - want[inner]).reshape(24, -1).max(axis=1)
    d_all = np.abs(got - want).reshape(24, -1).max(axis=1)
    scale = np.abs(want).reshape(24, -1).max(axis=1)
    bound = 379.0 * d_in + 1e-13 * np.maximum(scale, 1e-3 * scale.max())
    assert (d_all <= bound).all(), dict(zip(O.FIELD_NAMES, d_all / np.maximum(bound, 1e-300)))
    assert t == 0.25


@pytest.mark.parametrize("shape", [(64, 13, 11), (64, 16, 12)])
@pytest.mark.parametrize("cfg_name", ["32x8x1/1", "32x4x1/1", "32x4x2/1", "32x2x2/2"])
def test_full_row_variants(torch_cuda, cfg_name, shape):
    """With n0 a multiple of 32 the 32-wide float64 configurations run the
    kernel whose warps share first differences across lanes for the mixed
    second differences (and, when n1 and n2 fill the blocks, rows share them
    through shared memory for D_y D_z): right-hand side (faces, edges,
    corners, every lane of the row, rows past n1 and n2 in partial blocks)
    against the oracle and against a plain every-stencil kernel (1e-13), and
    RK4 steps against the oracle."""
    from paper_1111_3344_gb300 import bssn as B
    # the puncture sits on a cell corner, half a cell from the nearest points;
    # (64, 16, 12) fills every block of every 32-wide shape, so the kernel
    # also shares first differences along z between rows (D_y D_z)
    h = 0.1
    case = dict(n=shape, xmin=(-3.2, -h * (shape[1] // 2), -h * (shape[2] // 2)), h=h, boundary="sommerfeld",
                conformal="W", punctures=[(0.8, 0.0, 0.0, 0.0)], shift="gamma-driver", eta=1.5, q_R=1.2)
    cfg = oracle_cfg(case)
    bg = O.initial_data(cfg, "bl", bl_params(case))
    st = inputs.random_state(19, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    names = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())]
    rhs = {}
    for name in (cfg_name, "64x4x1/1"):  # the row variant and a plain (every-stencil) shape
        evo = _evo(case)
        B.bssn_set_tile(evo.ctx, names.index(name))
        rhs[name] = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
        evo.close()
    want, mag = O.rhs_mag(cfg, st)
    e = normwise_errors(rhs[cfg_name], want)
    e_plain = normwise_errors(rhs["64x4x1/1"], want)
    d = normwise_errors(rhs[cfg_name], rhs["64x4x1/1"])
    # Half a cell from the puncture the K and At right-hand sides are small
    # differences of much larger terms: the bar is 1e-12 of the larger of the
    # field's scale and the oracle's magnitude of the terms at the point
    # (rounding_aware_errors); normwise, trK measured 1.08e-12 for both kernels
    r = rounding_aware_errors(rhs[cfg_name], want, mag, TOL_RHS)
    r_plain = rounding_aware_errors(rhs["64x4x1/1"], want, mag, TOL_RHS)
    assert r.max() <= 1.0 and r_plain.max() <= 1.0, (dict(zip(O.FIELD_NAMES, r)), dict(zip(O.FIELD_NAMES, e)))
    assert e.max() <= 1.01 * e_plain.max() + 1e-15, (e.max(), e_plain.max())
    # same arithmetic but for the mixed-difference rounding (1/(12h) twice
    # instead of 1/(144h^2) once)
    assert d.max() <= 1e-13, dict(zip(O.FIELD_NAMES, d))
    evo = _evo(case)
    B.bssn_set_tile(evo.ctx, names.index(cfg_name))
    evo.set_state(st, 0.0)
    evo.rk4_step(2)
    e = normwise_errors(evo.get_state()[0], O.rk4(cfg, st, 2))
    assert e.max() <= TOL_STEP, dict(zip(O.FIELD_NAMES, e))
    evo.close()
