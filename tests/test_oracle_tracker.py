"""Pins for the oracle's puncture tracker (the paper's Sec. "Object tracking":
dx^i/dt = -beta^i at the puncture, shift interpolated to the puncture,
forward Euler).

* The interpolation reproduces every polynomial of degree <= 3 in each
  coordinate separately (tricubic), anywhere in the stored block, including
  next to and inside the ghost layers where the stencil is shifted.
* It returns the stored value at a grid point (to the rounding of the
  position), and misses a quartic.
* On a smooth function its error falls at fourth order.
* With a linear shift beta^i = -lam (x^i - c^i) the exact motion is
  x(t) = c + (x0 - c) e^{lam t}: the Euler track converges to it at first
  order in dt and moves away from c for lam > 0 (the sign of the law)."""
import itertools

import numpy as np
import pytest

import oracle as O


def _cfg(n=(10, 9, 11), h=0.2, xmin=(-1.0, -0.7, -1.2)):
    return O.Config(n=n, h=h, xmin=xmin, periodic=False)


def _mesh(cfg):
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    return Xc, Yc, Zc


def _stored_box(cfg):
    lo = [cfg.coords(d)[0] for d in range(3)]
    hi = [cfg.coords(d)[-1] for d in range(3)]
    return np.array(lo), np.array(hi)


@pytest.mark.parametrize("e", list(itertools.product(range(4), repeat=3))[::3])
def test_tricubic_exact(e):
    cfg = _cfg()
    X, Y, Z = _mesh(cfg)
    f = (X - 0.3) ** e[0] * (Y + 0.1) ** e[1] * (Z - 0.2) ** e[2] + 0.7 * X ** 3 * Z ** 2 - Y ** 3 + 2.0
    rng = np.random.default_rng(sum(e))
    lo, hi = _stored_box(cfg)
    for _ in range(20):
        p = lo + rng.random(3) * (hi - lo)
        want = (p[0] - 0.3) ** e[0] * (p[1] + 0.1) ** e[1] * (p[2] - 0.2) ** e[2] + 0.7 * p[0] ** 3 * p[2] ** 2 \
            - p[1] ** 3 + 2.0
        assert O.interp(cfg, f, p) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_grid_point_and_quartic():
    cfg = _cfg()
    X, Y, Z = _mesh(cfg)
    f = np.sin(X + 2 * Y) * np.cos(Z)
    for (i, j, k) in [(4, 5, 6), (1, 1, 1), (12, 10, 13), (8, 3, 9)]:
        p = [cfg.coords(0)[i], cfg.coords(1)[j], cfg.coords(2)[k]]
        # the position maps back to the node to rounding, so the value does too
        assert O.interp(cfg, f, p) == pytest.approx(f[k, j, i], rel=1e-13, abs=1e-15)
    q = X ** 4
    p = [0.13, 0.05, -0.31]
    assert abs(O.interp(cfg, q, p) - p[0] ** 4) > 1e-6


def test_fourth_order_convergence():
    errs = []
    rng = np.random.default_rng(7)
    pts = rng.random((30, 3)) * 0.8 - 0.4
    for h in (0.1, 0.05):
        n = int(round(2.0 / h))
        cfg = _cfg(n=(n, n, n), h=h, xmin=(-1.0, -1.0, -1.0))
        X, Y, Z = _mesh(cfg)
        f = np.sin(2 * X - Y) * np.exp(0.5 * Z)
        errs.append(max(abs(O.interp(cfg, f, p) - np.sin(2 * p[0] - p[1]) * np.exp(0.5 * p[2])) for p in pts))
    ratio = errs[0] / errs[1]
    assert 12.0 < ratio < 20.0, (errs, ratio)


def _linear_shift_state(cfg, lam, c):
    X, Y, Z = _mesh(cfg)
    st = np.zeros(cfg.shape)
    for d, V in enumerate((X, Y, Z)):
        st[O.F_BETA + d] = -lam * (V - c[d])
    return st


def test_euler_track_against_closed_form():
    cfg = _cfg(n=(20, 20, 20), h=0.1, xmin=(-1.0, -1.0, -1.0))
    lam, c, x0, T = 0.8, np.array([0.05, -0.1, 0.02]), np.array([0.15, 0.0, -0.05]), 0.5
    st = _linear_shift_state(cfg, lam, c)
    exact = c + (x0 - c) * np.exp(lam * T)
    errs = []
    for nsteps in (20, 40, 80):
        dt = T / nsteps
        pos = np.array([[1.0, *x0]])
        for _ in range(nsteps):
            pos = O.track_step(cfg, st, pos, dt)
        # Euler on a linear law: c + (x0 - c)(1 + lam dt)^n
        np.testing.assert_allclose(pos[0, 1:], c + (x0 - c) * (1 + lam * dt) ** nsteps, rtol=1e-12, atol=1e-14)
        assert pos[0, 0] == 1.0
        errs.append(np.abs(pos[0, 1:] - exact).max())
    assert np.linalg.norm(pos[0, 1:] - c) > np.linalg.norm(x0 - c)  # moves away from c
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2, errs


def test_several_punctures_independent():
    cfg = _cfg(n=(12, 12, 12), h=0.2, xmin=(-1.2, -1.2, -1.2))
    X, Y, Z = _mesh(cfg)
    st = np.zeros(cfg.shape)
    st[O.F_BETA] = 0.3 * X * Y
    st[O.F_BETA + 1] = Z ** 2 - 0.1
    st[O.F_BETA + 2] = X ** 3
    P = np.array([[1.0, 0.1, 0.2, -0.3], [0.5, -0.6, 0.45, 0.7], [0.2, 1.1, -1.0, 0.0]])
    out = O.track_step(cfg, st, P, 0.05)
    for a in range(3):
        x, y, z = P[a, 1:]
        want = np.array([x - 0.05 * 0.3 * x * y, y - 0.05 * (z * z - 0.1), z - 0.05 * x ** 3])
        np.testing.assert_allclose(out[a, 1:], want, rtol=1e-12, atol=1e-13)
        assert out[a, 0] == P[a, 0]
