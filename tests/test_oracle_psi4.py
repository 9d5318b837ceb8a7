"""Pins for the oracle's Weyl scalar Psi4 (the paper's Sec. "Gravitational
Waves", WeylScal4 with the fiducial tetrad).

* Exact spacetimes: tests/exact_solutions.psi4_exact contracts the exact
  4-Riemann tensor (Taylor jets of the 4-metric in grid coordinates, no 3+1
  split of the curvature) with the fiducial tetrad.  The oracle's Psi4 (Gauss,
  Codazzi and Ricci projections from 4th-order stencils of the ADM fields)
  converges to it at 4th order on Schwarzschild seen from a wavy grid, at and
  away from the grid origin, where Psi4 != 0 because the grid's radial
  direction is not a principal one, and in slices boosted against the
  Kerr-Schild ones, where the Codazzi projection (magnetic part) is non-zero
  too; it converges to 0 on flat space in wavy
  coordinates, where each of the three projections vanishes separately; on
  the gauge wave (metric and K depending on x alone) it is 0 to rounding.
* Flat metric with an extrinsic curvature K_ij linear in the coordinates: the
  3-curvature vanishes and the stencils are exact, so Psi4 has the closed form
  of the K terms contracted with the spherical unit vectors
  r = x/|x|, theta = (xz, yz, -rho^2)/(rho |x|), phi = (-y, x, 0)/rho.
* On the z axis the triad is undefined and Psi4 is 0."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O


def _mesh(cfg):
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    return Xc, Yc, Zc


BOXES = {"ks_wavy": (1.5, 2.5), "ks_offset": (1.5, 2.5), "ks_boost": (1.5, 2.5), "flat_wavy": (-0.5, 0.5),
         "gauge_wave": (-0.5, 0.5)}
INNER = (slice(3, -3),) * 3


@pytest.mark.parametrize("use_w", [True, False])
@pytest.mark.parametrize("name", ["ks_wavy", "ks_offset", "ks_boost", "flat_wavy", "gauge_wave"])
def test_psi4_exact_spacetimes(name, use_w):
    lo, hi = BOXES[name]
    errs = []
    for n in (12, 24):
        cfg = O.Config(n=(n, n, n), h=(hi - lo) / n, xmin=(lo,) * 3, periodic=name == "gauge_wave", use_w=use_w)
        X, Y, Z = _mesh(cfg)
        st, _, _ = E.on_grid(name, (n, n, n), lo, hi, use_w=use_w)
        got = O.psi4(cfg, st)
        # the exact value (jets of the 4-metric) at a seeded sample of 400
        # interior points, the corners of the interior block included
        rng = np.random.default_rng(n)
        k = np.concatenate([rng.integers(3, n + 3, 392), [3, 3, 3, 3, n + 2, n + 2, n + 2, n + 2]])
        j = np.concatenate([rng.integers(3, n + 3, 392), [3, 3, n + 2, n + 2, 3, 3, n + 2, n + 2]])
        i = np.concatenate([rng.integers(3, n + 3, 392), [3, n + 2, 3, n + 2, 3, n + 2, 3, n + 2]])
        want = E.psi4_exact(name, X[k, j, i], Y[k, j, i], Z[k, j, i])
        g = got[0][k, j, i] + 1j * got[1][k, j, i]
        errs.append(np.abs(g - want).max())
        scale = np.abs(want).max()
    ratio = errs[0] / errs[1]
    if name == "gauge_wave":
        # the metric and K depend on x alone: every discrete projection
        # vanishes algebraically, so Psi4 is zero to rounding at any h
        assert scale < 1e-12 and max(errs) < 1e-11, errs
        return
    if name.startswith("ks"):
        assert scale > {"ks_wavy": 5e-5, "ks_offset": 5e-3, "ks_boost": 5e-3}[name]  # Psi4 is non-zero here
        assert errs[1] < 1e-2 * scale, (errs, scale)
    else:
        assert scale < 1e-12  # flat: exactly zero
        assert errs[1] < 1e-3
    assert 11.0 < ratio < 22.0, (name, errs, ratio)


def _sph(X, Y, Z):
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rho = np.sqrt(X * X + Y * Y)
    rh = np.array([X, Y, Z]) / r
    th = np.array([X * Z, Y * Z, -rho * rho]) / (rho * r)
    ph = np.array([-Y, X, np.zeros_like(X)]) / rho
    return rh, th, ph


def test_psi4_flat_metric_linear_K_closed_form():
    cfg = O.Config(n=(10, 9, 8), h=0.23, xmin=(0.3, -1.1, -0.9), periodic=False, use_w=True)
    X, Y, Z = _mesh(cfg)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3)) * 0.3
    A = A + A.T                                 # K_ij = A_ij + B_ijk x^k
    B = rng.normal(size=(3, 3, 3)) * 0.2
    B = B + B.transpose(1, 0, 2)
    xs = np.array([X, Y, Z])
    K = A[:, :, None, None, None] + np.einsum("ijk,k...->ij...", B, xs)
    st = np.zeros(cfg.shape)
    st[O.F_CHI] = 1.0
    st[O.F_ALP] = 1.0
    sym = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for m, (i, j) in enumerate(sym):
        st[O.F_GT + m] = 1.0 if i == j else 0.0
    trK = K[0, 0] + K[1, 1] + K[2, 2]
    st[O.F_TRK] = trK
    for m, (i, j) in enumerate(sym):
        st[O.F_AT + m] = K[i, j] - (trK / 3.0 if i == j else 0.0)
    got = O.psi4(cfg, st)
    # closed form with the spherical triad; dK[k][j][l] = B_jlk
    Xi, Yi, Zi = X[INNER], Y[INNER], Z[INNER]
    Ki = K[(slice(None), slice(None)) + INNER]
    rh, th, ph = _sph(Xi, Yi, Zi)
    s2 = 1 / np.sqrt(2)
    n = -s2 * rh
    mb = s2 * (th - 1j * ph)
    Rs = np.einsum("ac...,bd...->abcd...", Ki, Ki) - np.einsum("ad...,bc...->abcd...", Ki, Ki)
    R0 = np.einsum("bdc->bcd", B) - np.einsum("bcd->bcd", B)  # D_c K_bd - D_d K_bc
    R00 = np.einsum("...,bd...->bd...", trK[INNER], Ki) - np.einsum("bm...,md...->bd...", Ki, Ki)
    want = (np.einsum("abcd...,a...,b...,c...,d...->...", Rs, n, mb, n, mb)
            + 2 * s2 * np.einsum("bcd,b...,c...,d...->...", R0, mb, n, mb)
            + 0.5 * np.einsum("bd...,b...,d...->...", R00, mb, mb))
    g = got[0][INNER] + 1j * got[1][INNER]
    np.testing.assert_allclose(g, want, rtol=1e-11, atol=1e-12)
    assert np.abs(want).max() > 0.1


def test_psi4_zero_on_z_axis():
    h = 0.2
    cfg = O.Config(n=(7, 7, 6), h=h, xmin=(-3.5 * h, -3.5 * h, 0.1), periodic=False, use_w=True)
    X, Y, Z = _mesh(cfg)
    st, _, _ = E.evaluate("flat_wavy", X, Y, Z + 0.0)
    got = O.psi4(cfg, st)
    # cell centres x = y = 0 exist: the middle column
    axis = (slice(3, -3), 3 + 3, 3 + 3)
    assert np.all(X[axis] == 0.0) and np.all(Y[axis] == 0.0)
    assert np.all(got[0][axis] == 0.0) and np.all(got[1][axis] == 0.0)
    off = (slice(3, -3), 3 + 2, 3 + 3)
    assert np.any(got[0][off] != 0.0)
