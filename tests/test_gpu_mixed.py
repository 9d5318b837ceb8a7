"""Mixed precision (float32 stencils and right-hand side, float64 RK4 state,
float64 W update near the puncture, float64 constraint reductions).

Tolerance of one right-hand side against the float64 oracle: float32 unit
roundoff 2^-24 = 6e-8 times the cancellation of the second-derivative
stencils, whose coefficients sum in magnitude to 64 against a result of order
h^2 f'': for the perturbed states here (h ~ 0.1-0.2, |f''|/|f| ~ 1-10) that
is 6e-8 x 64 / (12 h^2 |f''/f|) ~ 1e-6..5e-5 of the field's scale; the bar is
2e-4 normwise.  After an evolution the float64 state carries only the float32
error of the increments dt k, so the constraint norms of the mixed run stay
within 1e-6 relative of the float64 run in L2 (the rounding noise is
uncorrelated with the truncation error and enters the root mean square at
second order)."""
import numpy as np
import pytest

import oracle as O
from cases import bl_params, gpu_params, normwise_errors, oracle_cfg
from paper_1111_3344_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_MIXED_RHS = 2e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


BL = dict(n=(37, 21, 19), xmin=(-4.1, -2.3, -2.2), h=0.2203, boundary="sommerfeld",
          punctures=[(1.0, 0.05, -0.02, 0.01)], r_excise=0.8, conformal="W")


@pytest.mark.parametrize("w_thr", [0.0, 0.3, 2.0])
def test_mixed_rhs_close_to_oracle(torch_cuda, w_thr):
    from paper_1111_3344_gb300.bssn import Evolution
    case = dict(BL, precision="mixed", w_fp64_threshold=w_thr)
    bg = O.initial_data(oracle_cfg(case), "bl", bl_params(case))
    st = inputs.random_state(7, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    evo = Evolution(gpu_params(case))
    got = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    want = O.rhs(oracle_cfg(case), st)
    e = normwise_errors(got, want)
    print("mixed rhs normwise errors", dict(zip(O.FIELD_NAMES, np.round(e, 9))))
    assert e.max() <= TOL_MIXED_RHS, dict(zip(O.FIELD_NAMES, e))


def test_mixed_w_fp64_branch_matches_fp64_w_rhs(torch_cuda):
    """Below the threshold the W right-hand side is float64: it then agrees with
    the float64 path to float32 input rounding of the other fields only."""
    from paper_1111_3344_gb300.bssn import Evolution
    case = dict(BL, precision="mixed", w_fp64_threshold=10.0)
    bg = O.initial_data(oracle_cfg(case), "bl", bl_params(case))
    st = inputs.random_state(3, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    evo = Evolution(gpu_params(case))
    got = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    want = O.rhs(oracle_cfg(case), st)
    e = normwise_errors(got, want)
    case32 = dict(case, w_fp64_threshold=0.0)
    evo32 = Evolution(gpu_params(case32))
    got32 = evo32.register_to_numpy(evo32.rhs(evo32.numpy_to_register(st)))
    e32 = normwise_errors(got32, want)
    assert e[0] <= e32[0]
    assert e[0] < 1e-5


def _run(precision, n=48, steps=20, w_thr=0.2):
    from paper_1111_3344_gb300.bssn import Evolution, Params
    L = 8.0
    h = 2 * L / n
    p = Params(n=(n,) * 3, xmin=(-L,) * 3, h=h, boundary="sommerfeld", conformal="W", slicing="1+log",
               shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * h, precision=precision,
               w_fp64_threshold=w_thr, r_excise=1.0)
    evo = Evolution(p)
    evo.set_initial_data("bl", [1, 1.0, 0.0, 0.0, 0.0])
    evo.rk4_step(steps)
    st, t = evo.get_state()
    return st, evo.constraints()


def test_mixed_evolution_tracks_fp64(torch_cuda):
    """Regression bars of the float right-hand side against float64 on a small
    puncture (20 steps at 48^3).  They record what this path reaches, not the
    1e-6 constraint-norm target: at 256^3 after 100 steps its excised norms
    differ from float64 by percents, and the double-word path is the form that
    meets 1e-6 (test_gpu_ff)."""
    st64, c64 = _run("fp64")
    stmx, cmx = _run("mixed")
    e = normwise_errors(stmx, st64)
    print("per-field normwise state error after 20 steps", dict(zip(O.FIELD_NAMES, e)))
    rel = np.abs(cmx - c64) / np.maximum(np.abs(c64), 1e-300)
    print("constraint norm relative differences", rel)
    assert e.max() < 1e-4
    # L2 norms: Hamiltonian over the whole grid within 1e-6 relative of the
    # float64 run (measured 9e-8); over the excised region, where H itself is
    # smallest, within 2e-6 (measured 1.03e-6 on this 48^3 case); the momentum
    # components, first derivatives of K_ij that carry the float32 rounding
    # noise of the increments, within 3e-6 (measured 3-4e-7)
    assert rel[0] < 1e-6, rel
    assert rel[8] < 2e-6, rel
    assert rel[[1, 2, 3, 9, 10, 11]].max() < 3e-6, rel
    assert rel.max() < 1e-4, rel


def test_mixed_periodic_gauge_wave_runs(torch_cuda):
    from paper_1111_3344_gb300.bssn import Evolution
    case = dict(n=(24, 24, 24), xmin=(-0.5,) * 3, h=1 / 24, boundary="periodic", conformal="W",
                slicing="harmonic", shift="frozen", precision="mixed")
    evo = Evolution(gpu_params(case))
    evo.set_initial_data("gauge_wave", [0.01, 1.0])
    evo.rk4_step(10)
    got, _ = evo.get_state()
    want = O.rk4(oracle_cfg(case), O.initial_data(oracle_cfg(case), "gauge_wave", [0.01, 1.0]), 10)
    e = normwise_errors(got, want)
    assert e.max() < 1e-5, e


def _evo(case):
    from paper_1111_3344_gb300.bssn import Evolution
    return Evolution(gpu_params(case))


def test_split_stage_matches_oracle_and_fused(torch_cuda):
    """Every split-stage variant (stencil pass into a derivative register,
    algebra pass reading it): its right-hand side is within the float bar of
    the oracle and within float rounding of the fused kernel, and two RK4
    steps agree with the fused kernel's."""
    from paper_1111_3344_gb300 import bssn as B
    case = dict(n=(64, 13, 37), xmin=(-3.2, -0.7, -1.8), h=0.1, boundary="sommerfeld", conformal="W",
                punctures=[(0.8, 0.0, 0.0, 0.0)], precision="mixed", w_fp64_threshold=0.2)
    cfg = oracle_cfg(case)
    bg = O.initial_data(cfg, "bl", bl_params(case))
    st = inputs.random_state(29, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    want = O.rhs(cfg, st)
    names = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())]
    res = {}
    for name in ["32x8x1/1"] + [n for n in names if n.startswith("split")]:
        evo = _evo(case)
        B.bssn_set_tile(evo.ctx, names.index(name))
        rhs = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
        evo.set_state(st, 0.0)
        evo.rk4_step(2)
        res[name] = (rhs, evo.get_state()[0])
        evo.close()
    fused_rhs, fused_step = res["32x8x1/1"]
    for name, (rhs, step) in res.items():
        # half a cell from the puncture the float right-hand side is 1.9e-4
        # (normwise) from the oracle for the fused kernel too: the float bar
        # next to a puncture is the one of the 128^3 mixed step, 5e-4
        e = normwise_errors(rhs, want)
        assert e.max() <= 5e-4, (name, dict(zip(O.FIELD_NAMES, e)))
        d = normwise_errors(rhs, fused_rhs)
        assert d.max() <= 1e-5, (name, dict(zip(O.FIELD_NAMES, d)))
        # two RK4 steps: float rounding of different operation orders, the
        # bar of the tile-configuration test
        assert normwise_errors(step, fused_step).max() <= 1e-4, name


def test_mixed_float64_ksum_option(torch_cuda):
    """ksum_fp64 keeps the weighted sum of the k of every field in float64
    (the other mixed arithmetic unchanged).  Three steps against the float64
    oracle within the mixed step bar; the k-sum form changes the state by no
    more than the float rounding of the k that it avoids (dt times float32
    unit roundoff times |k| per step, below the mixed step bar); and a
    batch refuses the option."""
    from paper_1111_3344_gb300 import bssn as B
    case = dict(BL, precision="mixed", w_fp64_threshold=0.3)
    cfg = oracle_cfg(case)
    bg = O.initial_data(cfg, "bl", bl_params(case))
    st = inputs.random_state(9, case["n"], case["xmin"], case["h"], amp=0.03, background=bg)
    want = O.rk4(cfg, st, 3)
    out = {}
    for ks in (False, True):
        p = gpu_params(case)
        p.ksum_fp64 = ks
        evo = B.Evolution(p)
        evo.set_state(st, 0.0)
        evo.rk4_step(3)
        out[ks] = evo.get_state()[0]
        evo.close()
    e = normwise_errors(out[True], want)
    print("mixed ksum_fp64 3 steps normwise", e.max())
    assert e.max() <= 5e-4, dict(zip(O.FIELD_NAMES, e))
    d = normwise_errors(out[True], out[False])
    assert 0 < d.max() <= 5e-4, d.max()
    p = gpu_params(case)
    p.ksum_fp64 = True
    b = B.Batch("mixed", pool_bytes=B.Batch.member_bytes(gpu_params(case)) + (16 << 20), max_members=2)
    with pytest.raises(B.BssnError):
        b.add(p)
    b.close()
