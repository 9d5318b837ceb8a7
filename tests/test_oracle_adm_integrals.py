"""Pins for the oracle's ADM mass and angular momentum volume integrals (the
paper's Sec. "Masses and Momenta", volume-integral form, vacuum).

On exact vacuum data the Hamiltonian constraint turns the mass integrand into
-(1/2 pi) d_i(gt^ij d_j psi) and the momentum constraint turns the J_i
integrand into (1/8 pi) eps_ijk d_l(x^j psi^6 At^l_k), psi = e^{phi}.
tests/exact_solutions.py evaluates those divergences exactly (Taylor jets),
so:

* the oracle's integrands (finite differences of the exact BSSN data)
  converge to them at fourth order on spacetimes where every term is
  non-zero (Schwarzschild seen from a wavy grid, flat space in wavy
  coordinates, the gauge wave), for both the phi and the W variant;
* the box sums converge at second order (midpoint rule) to the outward flux
  through the box faces, integrated by Gauss-Legendre quadrature;
* conformally flat, time-symmetric data (Brill-Lindquist) have identically
  zero integrands, and the excised sums drop exactly the excised points.

A dropped term, a wrong power of psi, a wrong sign or a transposed index
breaks the fourth-order agreement on at least one of these spacetimes."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O


def _mesh(cfg):
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    return Xc, Yc, Zc


def _case(name, n, use_w, box):
    lo, hi = box
    cfg = O.Config(n=(n, n, n), h=(hi - lo) / n, xmin=(lo,) * 3, periodic=name == "gauge_wave",
                   use_w=use_w)
    st, _, grad = E.on_grid(name, (n, n, n), lo, hi, use_w=use_w)
    return cfg, st, grad


BOXES = {"ks_wavy": (1.5, 2.5), "flat_wavy": (-0.5, 0.5), "gauge_wave": (-0.5, 0.5)}


@pytest.mark.parametrize("use_w", [True, False])
@pytest.mark.parametrize("name", ["ks_wavy", "flat_wavy", "gauge_wave"])
def test_integrands_fourth_order(name, use_w):
    errs, scales = [], []
    for n in (12, 24):
        cfg, st, grad = _case(name, n, use_w, BOXES[name])
        _, dens = O.adm_integrals(cfg, st)
        inner = (slice(3, -3),) * 3
        want = np.concatenate([grad["M_dens"][None][(slice(None),) + inner],
                               grad["J_dens"][(slice(None),) + inner]])
        got = dens[(slice(None),) + inner]
        errs.append(np.abs(got - want).reshape(4, -1).max(axis=1))
        scales.append(np.abs(want).reshape(4, -1).max(axis=1))
    e0, e1 = errs
    live = scales[1] > 1e-6 * scales[1].max()  # components that are not identically zero
    assert live.any()
    ratio = e0[live] / np.maximum(e1[live], 1e-300)
    assert (ratio > 11.0).all() and (ratio < 22.0).all(), (name, ratio)
    assert (e1[live] < 1e-3 * scales[1][live]).all(), (e1, scales[1])


def _gauss_faces(lo, hi, m=10):
    """Points and weights of an m x m Gauss-Legendre rule on each face of the
    cube [lo, hi]^3, with the face's outward normal axis and sign."""
    t, w = np.polynomial.legendre.leggauss(m)
    s = lo + (t + 1) * (hi - lo) / 2
    ws = w * (hi - lo) / 2
    A, B = np.meshgrid(s, s, indexing="ij")
    W2 = np.outer(ws, ws)
    for axis in range(3):
        for sign, c in ((-1.0, lo), (1.0, hi)):
            pts = [None, None, None]
            others = [d for d in range(3) if d != axis]
            pts[axis] = np.full_like(A, c)
            pts[others[0]] = A
            pts[others[1]] = B
            yield axis, sign, pts, W2


def _surface_integrals(name, lo, hi):
    out = np.zeros(4)
    for axis, sign, (X, Y, Z), W2 in _gauss_faces(lo, hi):
        _, _, grad = E.evaluate(name, X, Y, Z)
        out[0] += sign * np.sum(W2 * grad["M_flux"][axis])
        for i in range(3):
            out[1 + i] += sign * np.sum(W2 * grad["J_flux"][i][axis])
    return out


@pytest.mark.parametrize("name", ["ks_wavy", "flat_wavy"])
def test_box_sums_converge_to_fluxes(name):
    lo, hi = BOXES[name]
    want = _surface_integrals(name, lo, hi)
    errs = []
    for n in (16, 32):
        cfg, st, _ = _case(name, n, True, (lo, hi))
        ints, _ = O.adm_integrals(cfg, st)
        # no punctures: the excised sums are the full sums
        np.testing.assert_array_equal(ints[:4], ints[4:])
        errs.append(np.abs(ints[:4] - want))
    scale = np.abs(want).max()
    live = np.abs(want) > 1e-3 * scale
    ratio = errs[0][live] / np.maximum(errs[1][live], 1e-300)
    assert (ratio > 3.0).all() and (ratio < 5.5).all(), (want, errs, ratio)
    assert (errs[1] < 1e-2 * scale).all(), (want, errs)


def test_brill_lindquist_zero_and_excision():
    """Conformally flat, time-symmetric data: At = K = 0, gt = delta (to the
    rounding of e^{-4 phi} gamma_ii) and Gt = 0, so both integrands vanish to
    rounding (the puncture's mass sits in the singular point, which the
    volume form does not see)."""
    p = [(1.0, 0.05, -0.1, 0.02), (0.5, 1.1, 0.3, -0.4)]
    cfg = O.Config(n=(16, 14, 12), h=0.25, xmin=(-2.0, -1.75, -1.5), periodic=False, use_w=True,
                   r_excise=0.6, punctures=p)
    st = O.initial_data(cfg, "bl", [2] + [v for q in p for v in q])
    ints, dens = O.adm_integrals(cfg, st)
    assert np.abs(dens).max() < 1e-12
    assert np.abs(ints).max() < 1e-12


def test_excised_sum_drops_points_near_punctures():
    """The excised sums equal the full sums minus h^3 times the integrands at
    the points within r_excise of a puncture (selected here independently)."""
    cfg, st, _ = _case("ks_wavy", 12, True, BOXES["ks_wavy"])
    cfg.punctures = [(1.0, 2.0, 2.1, 1.9), (0.3, 1.55, 2.45, 2.0)]
    cfg.r_excise = 0.3
    ints, dens = O.adm_integrals(cfg, st)
    X, Y, Z = _mesh(cfg)
    near = np.zeros(X.shape, bool)
    for (_, px, py, pz) in cfg.punctures:
        near |= np.sqrt((X - px) ** 2 + (Y - py) ** 2 + (Z - pz) ** 2) <= cfg.r_excise
    inner = np.zeros(X.shape, bool)
    inner[3:-3, 3:-3, 3:-3] = True
    assert (near & inner).sum() > 10
    vol = cfg.h ** 3
    full = dens[:, inner].sum(axis=1) * vol
    kept = dens[:, inner & ~near].sum(axis=1) * vol
    np.testing.assert_allclose(ints[:4], full, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(ints[4:], kept, rtol=1e-12, atol=1e-15)
