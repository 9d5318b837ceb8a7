"""Pins for the oracle's finite-difference operators (the paper's Sec.
"Spacetime Curvature Evolution": fourth-order finite differences, fifth-order
Kreiss-Oliger dissipation).

A fourth-order first- or second-derivative stencil is exact on polynomials of
degree <= 4; the upwind (lopsided) stencil likewise, on either side; the KO
sixth difference annihilates degree <= 5 and maps the grid's highest mode
(-1)^i to -64 (-1)^i per axis, so that +eps/(64h) times it damps that mode.
A wrong coefficient, sign, offset or axis fails one of these."""
import itertools

import numpy as np
import pytest

import oracle as O


def _grid(n=(7, 6, 5), h=0.37):
    cfg = O.Config(n=n, h=h, xmin=(-1.1, 0.4, 2.0))
    Xc, Yc, Zc = cfg.coords(0), cfg.coords(1), cfg.coords(2)
    Z, Y, X = np.meshgrid(Zc, Yc, Xc, indexing="ij")
    return cfg, (X, Y, Z)


def _interior(cfg, a):
    g = O.GHOST
    return a[g:g + cfg.n[2], g:g + cfg.n[1], g:g + cfg.n[0]]


MONOMIALS = [e for e in itertools.product(range(5), repeat=3) if sum(e) <= 4]


def _mono(XYZ, e):
    X, Y, Z = XYZ
    return X ** e[0] * Y ** e[1] * Z ** e[2]


def _dmono(XYZ, e, axes):
    """Exact derivative of the monomial along the listed axes."""
    e = list(e)
    coef = 1.0
    for a in axes:
        coef *= e[a]
        e[a] -= 1
        if e[a] < 0:
            return np.zeros_like(XYZ[0])
    return coef * _mono(XYZ, e)


@pytest.mark.parametrize("e", MONOMIALS)
def test_first_derivative_exact_on_degree4(e):
    cfg, XYZ = _grid()
    f = _mono(XYZ, e)
    for a in range(3):
        got = _interior(cfg, O.apply_stencil(cfg, "d1", f, a))
        want = _interior(cfg, _dmono(XYZ, e, [a]))
        np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("e", MONOMIALS)
def test_second_derivatives_exact_on_degree4(e):
    cfg, XYZ = _grid()
    f = _mono(XYZ, e)
    for a in range(3):
        for b in range(3):
            got = _interior(cfg, O.apply_stencil(cfg, "dd", f, a, b))
            want = _interior(cfg, _dmono(XYZ, e, [a, b]))
            np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-8)


@pytest.mark.parametrize("e", MONOMIALS)
@pytest.mark.parametrize("sign", [1.0, -1.0, 0.0])
def test_upwind_exact_on_degree4(e, sign):
    cfg, XYZ = _grid()
    f = _mono(XYZ, e)
    for a in range(3):
        got = _interior(cfg, O.apply_stencil(cfg, "up", f, a, sign=sign))
        want = _interior(cfg, _dmono(XYZ, e, [a]))
        np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-9)


def test_upwind_is_lopsided_toward_the_shift_sign():
    """beta >= 0 reads points -1..+3, beta < 0 reads -3..+1: a spike placed at
    offset +3 only reaches the centre through the beta >= 0 stencil."""
    cfg, XYZ = _grid(n=(9, 9, 9), h=1.0)
    f = np.zeros(cfg.shape[1:])
    g = O.GHOST
    c = g + 4
    f[c, c, c + 3] = 1.0
    pos = O.apply_stencil(cfg, "up", f, 0, sign=1.0)[c, c, c]
    neg = O.apply_stencil(cfg, "up", f, 0, sign=-1.0)[c, c, c]
    assert pos == pytest.approx(1.0 / 12.0)
    assert neg == 0.0
    f[:] = 0.0
    f[c, c, c - 3] = 1.0
    pos = O.apply_stencil(cfg, "up", f, 0, sign=1.0)[c, c, c]
    neg = O.apply_stencil(cfg, "up", f, 0, sign=-1.0)[c, c, c]
    assert pos == 0.0
    assert neg == pytest.approx(-1.0 / 12.0)


@pytest.mark.parametrize("e", [e for e in itertools.product(range(6), repeat=3) if sum(e) <= 5])
def test_ko_annihilates_degree5(e):
    cfg, XYZ = _grid(h=0.5)
    f = _mono(XYZ, e)
    got = _interior(cfg, O.apply_stencil(cfg, "ko", f))
    scale = np.abs(f).max() * 64
    assert np.abs(got).max() <= 1e-12 * scale


def test_ko_damps_highest_mode():
    cfg, XYZ = _grid(n=(8, 8, 8), h=0.25)
    shp = cfg.shape[1:]
    k, j, i = np.meshgrid(*(np.arange(s) for s in shp), indexing="ij")
    for axis, idx in enumerate((i, j, k)):
        f = (-1.0) ** idx
        got = _interior(cfg, O.apply_stencil(cfg, "ko", f))
        np.testing.assert_array_equal(got, _interior(cfg, -64.0 * f))
    f = (-1.0) ** (i + j + k)
    got = _interior(cfg, O.apply_stencil(cfg, "ko", f))
    np.testing.assert_array_equal(got, _interior(cfg, -3 * 64.0 * f))


def test_fourth_order_truncation_of_d1():
    """On a non-polynomial function the D1 error falls 16x per halving of h."""
    errs = []
    for n in (16, 32):
        cfg = O.Config(n=(n, 4, 4), h=1.0 / n, xmin=(0.0, 0.0, 0.0))
        X = cfg.coords(0)[None, None, :] * np.ones(cfg.shape[1:])
        f = np.sin(2 * np.pi * X)
        got = _interior(cfg, O.apply_stencil(cfg, "d1", f, 0))
        want = _interior(cfg, 2 * np.pi * np.cos(2 * np.pi * X))
        errs.append(np.abs(got - want).max())
    assert 14.0 < errs[0] / errs[1] < 17.0
