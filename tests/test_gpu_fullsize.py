"""Parity at the benchmark size: single Brill-Lindquist puncture, 128^3 on
[-8, 8]^3, W, 1+log, Gamma-driver eta = 2, Sommerfeld boundary, dt = 0.25 h,
in the launch configuration bench.py times (autotuned tiles).

* initial data: every stored point against the oracle;
* one right-hand side of a perturbed state: sampled points (interior, faces,
  edges, corners, next to the puncture) against the oracle point by point;
* one RK4 step of the puncture data: every point against the oracle's full
  step (a few seconds of host work);
* the mixed path's RK4 step against the same oracle step, within the mixed
  tolerance."""
import numpy as np
import pytest

import oracle as O
from cases import normwise_errors, rounding_aware_errors
from paper_1111_3344_gb300 import inputs

pytestmark = pytest.mark.gpu

N, L = 128, 8.0
H = 2 * L / N
BL = [1, 1.0, 0.0, 0.0, 0.0]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


def _params(precision="fp64"):
    from paper_1111_3344_gb300.bssn import Params
    return Params(n=(N,) * 3, xmin=(-L,) * 3, h=H, boundary="sommerfeld", conformal="W", slicing="1+log",
                  shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * H, precision=precision,
                  w_fp64_threshold=0.2, r_excise=1.0)


def _cfg():
    return O.Config(n=(N,) * 3, xmin=(-L,) * 3, h=H, periodic=False, use_w=True, slicing="1+log",
                    shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * H, r_excise=1.0,
                    punctures=[(1.0, 0.0, 0.0, 0.0)])


@pytest.fixture(scope="module")
def oracle_id():
    return O.initial_data(_cfg(), "bl", BL)


def _evo(precision="fp64"):
    from paper_1111_3344_gb300 import bssn as B
    evo = B.Evolution(_params(precision))
    evo.set_initial_data("bl", BL)
    B.bssn_autotune(evo.ctx, reps=1)
    return evo


def test_fullsize_initial_data(torch_cuda, oracle_id):
    evo = _evo()
    got, _ = evo.get_state()
    assert normwise_errors(got, oracle_id).max() <= 1e-13
    evo.close()


def _sample_points(rng, count=1500):
    S = N + 6
    pts = [rng.integers(0, S, size=3) for _ in range(count)]
    # faces, edges, corners of every layer, and the points next to the puncture
    for a in (0, 1, 2, 3, S - 4, S - 3, S - 2, S - 1):
        for b in (0, 2, S // 2, S - 1):
            pts += [(a, b, S // 3), (b, a, 7), (9, b, a), (a, a, b), (a, b, a)]
    c = 3 + N // 2
    pts += [(c + i, c + j, c + k) for i in (-2, -1, 0, 1) for j in (-1, 0) for k in (-1, 0)]
    return np.array(pts, dtype=np.int32)


def test_fullsize_rhs_sampled(torch_cuda, oracle_id):
    st = inputs.random_state(44, (N,) * 3, (-L,) * 3, H, amp=0.02, background=oracle_id)
    evo = _evo()
    got = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    ijk = _sample_points(np.random.default_rng(1), count=4000)
    want, mag = O.rhs_points_mag(_cfg(), st, ijk)              # (P, 24), oracle
    g = np.stack([got[:, k, j, i] for (i, j, k) in ijk])       # (P, 24), CUDA path
    # normwise per field over the sample (which includes the points next to
    # the puncture, where every field takes its largest values)
    err = normwise_errors(g.T, want.T)
    print("full-size rhs normwise errors", dict(zip(O.FIELD_NAMES, err)))
    # Half a cell from the puncture the K and At right-hand sides are small
    # differences of terms ~1e3 times larger (W^2 times the lapse Laplacian
    # against 2 W^2 grad(phi).grad(alpha), with grad(phi) ~ 1/r), so two float64
    # evaluations that round in a different order differ there by a few ulp
    # of those terms (normwise 2.7e-12 in trK).  The bar is therefore 1e-12 of
    # the larger of the field's scale and the oracle's magnitude of the terms
    # at the point (cases.rounding_aware_errors).
    r = rounding_aware_errors(g.T, want.T, mag.T)
    print("full-size rhs rounding-aware ratios", dict(zip(O.FIELD_NAMES, r)))
    assert r.max() <= 1.0, dict(zip(O.FIELD_NAMES, r))
    # away from the cancellation the plain normwise bar holds as well
    away = [O.F_CHI] + list(range(O.F_GT, O.F_GT + 6)) + [O.F_ALP] + list(range(O.F_BETA, 24))
    assert err[away].max() <= 1e-12, dict(zip(O.FIELD_NAMES, err))
    evo.close()


@pytest.fixture(scope="module")
def oracle_step(oracle_id):
    return O.rk4(_cfg(), oracle_id, 1)


def test_fullsize_rk4_step_fp64(torch_cuda, oracle_step):
    evo = _evo("fp64")
    evo.rk4_step(1)
    got, t = evo.get_state()
    e = normwise_errors(got, oracle_step)
    assert e.max() <= 1e-11, dict(zip(O.FIELD_NAMES, e))
    assert t == pytest.approx(0.25 * H)
    evo.close()


def test_fullsize_rk4_step_mixed(torch_cuda, oracle_step):
    """One mixed-precision step against the float64 oracle step: the state
    error is dt times the float32 error of the k's; fields that start at zero
    (beta, B) are normalised by the floor of the metric, so their bound is the
    loosest: 5e-4 normwise."""
    evo = _evo("mixed")
    evo.rk4_step(1)
    got, _ = evo.get_state()
    e = normwise_errors(got, oracle_step)
    print("full-size mixed step normwise errors", dict(zip(O.FIELD_NAMES, e)))
    assert e.max() <= 5e-4, dict(zip(O.FIELD_NAMES, e))
    evo.close()
