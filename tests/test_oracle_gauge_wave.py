"""Pins for the gauge-wave workload (24^3 periodic grid on [-0.5, 0.5]^3,
A = 0.01, wavelength 1, harmonic slicing, zero shift, KO eps = 0.1,
dt = 0.25 dx, 50 steps): the oracle's initial data equal the exact solution
(tests/exact_solutions.py, built independently from the 4-metric), and the
full RK4 evolution converges to the exact solution at fourth order.  The wave
depends on x only, so the convergence runs use quasi-one-dimensional grids
(N x 4 x 4 points) that hold the same discrete solution."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O


def _cfg(n, ny=4):
    return O.Config(n=(n, ny, ny), h=1.0 / n, xmin=(-0.5, -0.5, -0.5), periodic=True,
                    use_w=True, slicing="harmonic", shift="frozen", ko_eps=0.1,
                    dt=0.25 / n)


def _exact(cfg, time):
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    st, _, _ = E.evaluate("gauge_wave", Xc, Yc, Zc, time=time)
    return st


def test_gauge_wave_initial_data_matches_exact_solution():
    cfg = _cfg(24, 24)
    st = O.initial_data(cfg, "gauge_wave", [0.01, 1.0])
    np.testing.assert_allclose(st, _exact(cfg, 0.0), rtol=0, atol=2e-15)


def test_gauge_wave_evolution_fourth_order():
    errs = []
    for n, steps in ((24, 50), (48, 100), (96, 200)):
        cfg = _cfg(n)
        st = O.initial_data(cfg, "gauge_wave", [0.01, 1.0])
        out = O.rk4(cfg, st, steps)
        t_end = steps * cfg.dt
        g = O.GHOST
        diff = (out - _exact(cfg, t_end))[:, g:-g, g:-g, g:-g]
        errs.append(np.abs(diff).max(axis=(1, 2, 3)))
    errs = np.array(errs)
    for f in (O.F_CHI, O.F_GT, O.F_GT + 3, O.F_TRK, O.F_AT, O.F_GAM, O.F_ALP):
        r = errs[:-1, f] / errs[1:, f]
        assert np.all(r > 12.0), (O.FIELD_NAMES[f], errs[:, f], r)
    assert errs[0].max() < 5e-5
