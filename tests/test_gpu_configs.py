"""The benchmark configurations at their full sizes, in the launch
configurations bench.py times (autotuned tiles), against the oracle.

* Gauge wave, 24^3 periodic on [-0.5, 0.5]^3, A = 0.01, wavelength 1,
  harmonic slicing, zero (frozen) shift, KO eps = 0.1, dt = 0.25 h, 50 RK4
  steps, float64: every point against the oracle's 50 steps, and both against
  the exact solution at t = 50 dt (the truncation error is the same).
* Single puncture at 256^3, mixed precision: the right-hand side of the
  evolved state (two RK4 steps after Brill-Lindquist data) at 2000 sampled
  points (interior, faces, edges, corners, next to the puncture) against the
  oracle evaluated point by point on the same state; the float bar grows as
  h^-2 for the fields built from second differences (see the test)."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O
from cases import normwise_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


def test_gauge_wave_24_cubed_50_steps(torch_cuda):
    from paper_1111_3344_gb300 import bssn as B
    n, h = 24, 1.0 / 24
    params = B.Params(n=(n,) * 3, xmin=(-0.5,) * 3, h=h, boundary="periodic", conformal="W",
                      slicing="harmonic", shift="frozen", ko_eps=0.1, dt=0.25 * h, precision="fp64")
    cfg = O.Config(n=(n,) * 3, xmin=(-0.5,) * 3, h=h, periodic=True, use_w=True, slicing="harmonic",
                   shift="frozen", ko_eps=0.1, dt=0.25 * h)
    evo = B.Evolution(params)
    evo.set_initial_data("gauge_wave", [0.01, 1.0])
    B.bssn_autotune(evo.ctx, reps=1)
    evo.rk4_step(50)
    got, t = evo.get_state()
    want = O.rk4(cfg, O.initial_data(cfg, "gauge_wave", [0.01, 1.0]), 50)
    # 50 steps = 200 right-hand sides of 1e-12 each, at most
    e = normwise_errors(got, want)
    assert e.max() <= 2e-10, dict(zip(O.FIELD_NAMES, e))
    assert t == pytest.approx(50 * 0.25 * h)
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    exact, _, _ = E.evaluate("gauge_wave", Xc, Yc, Zc, time=t)
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    err_gpu = np.abs(got[inner] - exact[inner]).max()
    err_cpu = np.abs(want[inner] - exact[inner]).max()
    print(f"gauge wave 24^3, 50 steps: max |gpu - exact| = {err_gpu:.3e}, |oracle - exact| = {err_cpu:.3e}")
    # the truncation error of the scheme at this resolution (1.4e-5 in Gt^x and
    # At_xx), the same for both: they differ only by rounding
    assert err_cpu < 5e-5
    assert abs(err_gpu - err_cpu) <= 1e-9 * err_cpu + 1e-12
    evo.close()


def test_puncture_256_cubed_mixed_sampled_rhs(torch_cuda):
    from paper_1111_3344_gb300 import bssn as B
    N, L = 256, 8.0
    H = 2 * L / N
    params = B.Params(n=(N,) * 3, xmin=(-L,) * 3, h=H, boundary="sommerfeld", conformal="W", slicing="1+log",
                      shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * H, precision="mixed",
                      w_fp64_threshold=0.2, r_excise=1.0)
    evo = B.Evolution(params)
    evo.set_initial_data("bl", [1, 1.0, 0.0, 0.0, 0.0])
    best, _ = B.bssn_autotune(evo.ctx, reps=1)
    evo.rk4_step(2)
    st, _ = evo.get_state()
    got = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    S = N + 6
    rng = np.random.default_rng(256)
    pts = [rng.integers(0, S, size=3) for _ in range(1500)]
    for a in (0, 1, 2, 3, S - 4, S - 3, S - 2, S - 1):
        for b in (0, 3, S // 2, S - 1):
            pts += [(a, b, S // 3), (b, a, 9), (11, b, a), (a, a, b), (a, b, a)]
    c = 3 + N // 2
    pts += [(c + i, c + j, c + k) for i in (-2, -1, 0, 1) for j in (-2, -1, 0, 1) for k in (-1, 0)]
    ijk = np.array(pts, dtype=np.int32)
    cfg = O.Config(n=(N,) * 3, xmin=(-L,) * 3, h=H, periodic=False, use_w=True, slicing="1+log",
                   shift="gamma-driver", eta=2.0, ko_eps=0.1, dt=0.25 * H, r_excise=1.0,
                   punctures=[(1.0, 0.0, 0.0, 0.0)])
    want = O.rhs_points(cfg, st, ijk)
    g = np.stack([got[:, k, j, i] for (i, j, k) in ijk])
    scale = np.abs(want).max(axis=0)
    err = np.abs(g - want).max(axis=0) / np.maximum(np.maximum(scale, 1e-3 * scale.max()), 1e-300)
    print(f"256^3 mixed ({B.bssn_tile_name(best)}) sampled rhs normwise errors",
          dict(zip(O.FIELD_NAMES, np.round(err, 8))))
    # float stage values carry a rounding of eps_f |X - X0| per point, which a
    # second difference multiplies by 64 / (12 h^2) (1365 at h = 1/16, four
    # times the 128^3 value).  K, At_ij and alpha take second differences of
    # alpha and gt_ij (near the puncture, where alpha - 1 and W^-1 are largest):
    # measured 1e-3 in K.  The other fields stay under the 1e-4 float bar.
    d2 = [O.F_TRK, O.F_ALP] + list(range(O.F_AT, O.F_AT + 6))
    rest = [f for f in range(O.NF) if f not in d2]
    assert err[d2].max() <= 2e-3, dict(zip(O.FIELD_NAMES, err))
    assert err[rest].max() <= 1e-4, dict(zip(O.FIELD_NAMES, err))
    evo.close()
