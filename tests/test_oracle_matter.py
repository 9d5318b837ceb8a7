"""Pins for the oracle's matter coupling (the paper's Sec. "Spacetime
Curvature Evolution" source terms with the projections E, S, S_i, S_ij of
T_{mu nu}, Sec. "TmunuBase").

The data are exact solutions of Einstein's equations with a perfect fluid:
spatially flat dust and radiation universes (a ~ t^{2/3}, t^{1/2},
rho = 3 H^2 / 8 pi) seen from tilted, curved, time-dependent coordinates
(tests/exact_solutions.py), so that E, S, S_i and the trace-free part of S_ij
are all non-zero on the slices and T_{mu nu} is the exact tensor pulled back
to the grid coordinates.

* With T_{mu nu} the right-hand sides of phi/W, gt, K, At and Gt converge at
  4th order to the exact time derivatives; without it K, At and Gt miss by
  O(1): the source terms are live, and their factors (4 pi, 8 pi, 16 pi) and
  signs are fixed by the exact solution, not by the printed formulas.
* The Hamiltonian and momentum constraints with the -16 pi E and -8 pi S_i
  terms converge to 0 at 4th order.
* The ADM mass and angular momentum integrands with the 16 pi E and
  8 pi x^j S_k terms converge to the exact divergences of the surface fluxes
  (the constraints with matter make them divergences again)."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O


def _setup(name, n, use_w):
    lo, hi = -0.5, 0.5
    cfg = O.Config(n=(n, n, n), h=(hi - lo) / n, xmin=(lo,) * 3, periodic=False, use_w=use_w)
    state, dts, grad = E.on_grid(name, (n, n, n), lo, hi, use_w=use_w)
    return cfg, state, dts, grad


INNER = (slice(3, -3),) * 3


def _rhs_errors(name, n, use_w, matter=True):
    cfg, state, dts, grad = _setup(name, n, use_w)
    if matter:
        cfg.tmunu = np.ascontiguousarray(grad["tmunu"])
    r = O.rhs(cfg, state)
    err = np.array([np.abs((r[f] - dts[f])[INNER]).max() for f in range(17)])
    scale = np.array([np.abs(dts[f][INNER]).max() for f in range(17)])
    return err, scale


@pytest.mark.parametrize("name", ["flrw_dust", "flrw_rad"])
@pytest.mark.parametrize("use_w", [True, False])
def test_rhs_with_matter_converges(name, use_w):
    e1, s1 = _rhs_errors(name, 12, use_w)
    e2, s2 = _rhs_errors(name, 24, use_w)
    assert (s1 > 1e-4).all(), s1
    ratio = e1 / np.maximum(e2, 1e-300)
    for f in range(17):
        assert e2[f] < 2e-4 * max(s2[f], 1.0), (O.FIELD_NAMES[f], e2[f], s2[f])
        assert ratio[f] > 12.0, (O.FIELD_NAMES[f], e1[f], e2[f], ratio[f])


@pytest.mark.parametrize("name", ["flrw_dust", "flrw_rad"])
def test_vacuum_rhs_misses_the_matter(name):
    """Dropping T_{mu nu} leaves K, At and Gt off by far more than the
    truncation error with it; phi/W and gt carry no source term."""
    ev, _ = _rhs_errors(name, 24, True, matter=False)
    em, _ = _rhs_errors(name, 24, True, matter=True)
    for f in [O.F_TRK] + list(range(O.F_AT, O.F_AT + 6)) + list(range(O.F_GAM, O.F_GAM + 3)):
        assert ev[f] > 10.0 * em[f], (O.FIELD_NAMES[f], ev[f], em[f])
    for f in [O.F_CHI] + list(range(O.F_GT, O.F_GT + 6)):
        assert ev[f] == em[f], O.FIELD_NAMES[f]


@pytest.mark.parametrize("name", ["flrw_dust", "flrw_rad"])
def test_constraints_with_matter_converge_to_zero(name):
    errs = []
    for n in (12, 24):
        cfg, state, _, grad = _setup(name, n, True)
        cfg.tmunu = np.ascontiguousarray(grad["tmunu"])
        _, H, M = O.constraints(cfg, state)
        errs.append(np.array([np.abs(H[INNER]).max()] + [np.abs(M[a][INNER]).max() for a in range(3)]))
        if n == 24:
            cfg.tmunu = None
            _, H0, _ = O.constraints(cfg, state)
            assert np.abs(H0[INNER]).max() > 1.0  # 16 pi E of a unit-scale universe
    ratio = errs[0] / errs[1]
    assert (ratio > 12.0).all(), (errs, ratio)
    assert (errs[1] < 1e-3).all(), errs


@pytest.mark.parametrize("name", ["flrw_dust", "flrw_rad"])
def test_adm_integrands_with_matter(name):
    errs = []
    for n in (12, 24):
        cfg, state, _, grad = _setup(name, n, True)
        cfg.tmunu = np.ascontiguousarray(grad["tmunu"])
        _, dens = O.adm_integrals(cfg, state)
        want = np.concatenate([grad["M_dens"][None], grad["J_dens"]])
        errs.append(np.abs(dens[(slice(None),) + INNER] - want[(slice(None),) + INNER]).reshape(4, -1).max(axis=1))
        scale = np.abs(want[(slice(None),) + INNER]).reshape(4, -1).max(axis=1)
    assert (scale > 1e-3).all(), scale
    ratio = errs[0] / errs[1]
    assert (ratio > 11.0).all(), (errs, ratio)
