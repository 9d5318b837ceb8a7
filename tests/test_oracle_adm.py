"""Pins for the oracle's general ADM -> BSSN conversion (the paper's Sec.
"Initial Conditions": BSSN variables by their definitions, B^i = 0, Gt^i from
derivatives of the metric, cubic extrapolation of Gt^i on the outer layers,
faces perpendicular, edges and corners along the summed normals, innermost
layer first).

* The extrapolation is exact for cubic polynomials, on every ghost point of
  every layer, face, edge and corner.
* On exact spacetimes in generic coordinates (ADM data from
  tests/exact_solutions.py) every non-Gt field equals the exact BSSN value
  to rounding, and Gt^i converges at fourth order to the exact Gt^i inside and
  on the extrapolated layers."""
import itertools

import numpy as np
import pytest

import exact_solutions as E
import oracle as O


def _mesh(cfg):
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    return Xc, Yc, Zc


@pytest.mark.parametrize("e", [e for e in itertools.product(range(4), repeat=3) if sum(e) <= 3])
def test_cubic_extrapolation_exact_on_cubics(e):
    cfg = O.Config(n=(6, 5, 7), h=0.3, xmin=(-1.0, 0.2, 0.5), periodic=False)
    X, Y, Z = _mesh(cfg)
    f = (X - 0.1) ** e[0] * (Y + 0.2) ** e[1] * Z ** e[2] + 0.5 * X * Y - 0.3 * Z ** 3 + 1.0
    g = f.copy()
    gh = np.ones(f.shape, bool)
    gh[3:-3, 3:-3, 3:-3] = False
    g[gh] = 1e30  # garbage in the ghosts: the result may not depend on it
    out = O.extrapolate_ghosts(cfg, g)
    np.testing.assert_allclose(out, f, rtol=1e-11, atol=1e-10)


def test_quartic_is_not_reproduced():
    """Extrapolation really is cubic: a quartic along x is missed on the x faces."""
    cfg = O.Config(n=(6, 6, 6), h=0.3, xmin=(-1.0, -1.0, -1.0), periodic=False)
    X, Y, Z = _mesh(cfg)
    f = X ** 4
    out = O.extrapolate_ghosts(cfg, f)
    assert np.abs(out - f).max() > 1e-3


@pytest.mark.parametrize("name,box", [("flat_wavy", (-0.5, 0.5)), ("ks_wavy", (1.5, 2.5))])
def test_adm_to_bssn_fd_on_exact_solutions(name, box):
    errs_in, errs_gh = [], []
    for n in (12, 24):
        lo, hi = box
        cfg = O.Config(n=(n, n, n), h=(hi - lo) / n, xmin=(lo,) * 3, periodic=False, use_w=True)
        X, Y, Z = _mesh(cfg)
        st_exact, _, grad = E.on_grid(name, (n, n, n), lo, hi)
        st = O.adm_to_bssn_fd(cfg, grad["adm"])
        # all non-Gt fields by the definitions, exactly; B^i = 0
        others = [f for f in range(O.F_B) if not O.F_GAM <= f < O.F_GAM + 3]
        np.testing.assert_allclose(st[others], st_exact[others], rtol=1e-12, atol=1e-13)
        assert np.all(st[O.F_B:] == 0.0)
        d = np.abs(st[O.F_GAM:O.F_GAM + 3] - st_exact[O.F_GAM:O.F_GAM + 3])
        inner = np.zeros(X.shape, bool)
        inner[3:-3, 3:-3, 3:-3] = True
        errs_in.append(d[:, inner].max())
        errs_gh.append(d[:, ~inner].max())
    assert errs_in[0] / errs_in[1] > 12.0, errs_in
    assert errs_in[1] < 1e-4
    if name == "ks_wavy":
        # three layers of cubic extrapolation converge at 4th order on smooth
        # data; flat_wavy's Gt has fourth derivatives ~1e3, which keeps its
        # extrapolated layers pre-asymptotic at these resolutions
        assert errs_gh[0] / errs_gh[1] > 10.0, errs_gh
        assert errs_gh[1] < 1e-3


def test_adm_to_bssn_fd_periodic_copies_ghosts():
    cfg = O.Config(n=(12, 12, 12), h=1 / 12, xmin=(-0.5,) * 3, periodic=True, use_w=False)
    X, Y, Z = _mesh(cfg)
    _, _, grad = E.evaluate("gauge_wave", X, Y, Z, use_w=False)
    st = O.adm_to_bssn_fd(cfg, grad["adm"])
    np.testing.assert_array_equal(st, O.fill_periodic(cfg, st))
