"""Pins for the oracle's constraint monitor (the paper's Sec. "Other analysis
modules": H = R - K^i_j K^j_i + K^2, M_i = nabla_j K_i^j - nabla_i K, vacuum).

* Conformally flat data gamma = psi^4 delta, K_ij = 0: H = -8 psi^-5 lap(psi)
  (closed form), converging at fourth order.
* Flat metric with an arbitrary smooth K_ij: H = K^2 - K^i_j K^j_i pointwise
  (no derivatives) and M_i = d_j K_ij - d_i K, the latter at fourth order.
* Exact vacuum solutions in generic coordinates: H = M_i = 0 up to O(h^4).
* Brill-Lindquist data (psi = 1 + sum m/(2r), K_ij = 0) solve H = 0 in the
  continuum; the excised L2 norm falls 16x per halving of h.
* The norm definitions (root mean square, maximum, excision) against the
  returned pointwise grids."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O


def _mesh(cfg):
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    return Xc, Yc, Zc


def _int(cfg, a):
    g = O.GHOST
    return a[..., g:g + cfg.n[2], g:g + cfg.n[1], g:g + cfg.n[0]]


def _bssn_from_psi_K(cfg, psi, Kij):
    """BSSN fields for gamma = psi^4 delta and the given K_ij (6 comps)."""
    st = np.zeros(cfg.shape)
    st[O.F_CHI] = psi ** -2 if cfg.use_w else np.log(psi)
    for m in (0, 3, 5):
        st[O.F_GT + m] = 1.0
    trK = (Kij[0] + Kij[3] + Kij[5]) / psi ** 4
    st[O.F_TRK] = trK
    for m in range(6):
        delta = 1.0 if m in (0, 3, 5) else 0.0
        st[O.F_AT + m] = psi ** -4 * (Kij[m] - psi ** 4 * delta * trK / 3)
    st[O.F_ALP] = 1.0
    return st


@pytest.mark.parametrize("use_w", [True, False])
def test_hamiltonian_conformally_flat_closed_form(use_w):
    errs = []
    for n in (16, 32):
        cfg = O.Config(n=(n, n, n), h=2.0 / n, xmin=(-1.0,) * 3, use_w=use_w)
        X, Y, Z = _mesh(cfg)
        a, kx, ky, kz = 0.2, 1.3, 0.7, 1.1
        psi = 1.0 + a * np.sin(kx * X) * np.cos(ky * Y) * np.sin(kz * Z + 0.3)
        lap = -(kx ** 2 + ky ** 2 + kz ** 2) * (psi - 1.0)
        Hex = -8.0 * psi ** -5 * lap
        st = _bssn_from_psi_K(cfg, psi, np.zeros((6,) + psi.shape))
        _, H, M = O.constraints(cfg, st)
        errs.append(np.abs(_int(cfg, H - Hex)).max())
        assert np.abs(_int(cfg, M)).max() < 1e-12
    assert errs[1] < 1e-4 and errs[0] / errs[1] > 13.0, errs


def test_flat_metric_arbitrary_K():
    errs = []
    for n in (16, 32):
        cfg = O.Config(n=(n, n, n), h=2.0 / n, xmin=(-1.0,) * 3, use_w=True)
        X, Y, Z = _mesh(cfg)
        K = np.stack([np.sin(X + 2 * Y), 0.3 * np.cos(Y - Z), 0.2 * np.sin(X * Z),
                      np.cos(Z) * np.sin(Y), 0.4 * np.sin(X - Y + Z), 0.5 + np.cos(2 * X)])
        st = _bssn_from_psi_K(cfg, np.ones_like(X), K)
        _, H, M = O.constraints(cfg, st)
        Km = np.array([[K[0], K[1], K[2]], [K[1], K[3], K[4]], [K[2], K[4], K[5]]])
        trK = K[0] + K[3] + K[5]
        KK = np.einsum("ij...,ji...->...", Km, Km)
        np.testing.assert_allclose(_int(cfg, H), _int(cfg, trK ** 2 - KK), rtol=1e-12, atol=1e-12)
        # d_j K_ij - d_i K, exact derivatives
        dK = {  # d/dx, d/dy, d/dz of each component
            0: (np.cos(X + 2 * Y), 2 * np.cos(X + 2 * Y), 0 * X),
            1: (0 * X, -0.3 * np.sin(Y - Z), 0.3 * np.sin(Y - Z)),
            2: (0.2 * Z * np.cos(X * Z), 0 * X, 0.2 * X * np.cos(X * Z)),
            3: (0 * X, np.cos(Z) * np.cos(Y), -np.sin(Z) * np.sin(Y)),
            4: (0.4 * np.cos(X - Y + Z), -0.4 * np.cos(X - Y + Z), 0.4 * np.cos(X - Y + Z)),
            5: (-2 * np.sin(2 * X), 0 * X, 0 * X),
        }
        sym = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]
        Mex = [sum(dK[sym[i][j]][j] for j in range(3)) - (dK[0][i] + dK[3][i] + dK[5][i])
               for i in range(3)]
        errs.append(max(np.abs(_int(cfg, M[i] - Mex[i])).max() for i in range(3)))
    assert errs[1] < 1e-4 and errs[0] / errs[1] > 13.0, errs


@pytest.mark.parametrize("name,box", [("flat_wavy", (-0.5, 0.5)), ("ks_wavy", (1.5, 2.5))])
def test_constraints_vanish_on_exact_solutions(name, box):
    errs = []
    for n in (12, 24):
        lo, hi = box
        cfg = O.Config(n=(n, n, n), h=(hi - lo) / n, xmin=(lo,) * 3, use_w=True)
        st, _, _ = E.on_grid(name, (n, n, n), lo, hi)
        _, H, M = O.constraints(cfg, st)
        errs.append([np.abs(_int(cfg, H)).max()] + [np.abs(_int(cfg, M[i])).max() for i in range(3)])
    errs = np.array(errs)
    assert (errs[0] / errs[1] > 12.0).all(), errs
    assert errs[1].max() < 1e-3


def test_brill_lindquist_hamiltonian_converges():
    l2 = []
    for n in (32, 64):
        cfg = O.Config(n=(n, n, n), h=8.0 / n, xmin=(-4.0,) * 3, periodic=False, use_w=True,
                       r_excise=1.0, punctures=[(1.0, 0.0, 0.0, 0.0)])
        st = O.initial_data(cfg, "bl", [1, 1.0, 0.0, 0.0, 0.0])
        norms, H, M = O.constraints(cfg, st)
        l2.append(norms[8])  # excised L2 of H
        assert norms[9:12].max() == 0.0  # K_ij = 0: M vanishes identically
    assert l2[0] / l2[1] > 13.0, l2


def test_norm_definitions():
    n = 16
    cfg = O.Config(n=(n, n, n), h=8.0 / n, xmin=(-4.0,) * 3, periodic=False, use_w=True,
                   r_excise=1.5, punctures=[(0.6, 0.7, 0.0, 0.0), (0.4, -1.05, 0.0, 0.0)])
    st = O.initial_data(cfg, "bl", [2, 0.6, 0.7, 0.0, 0.0, 0.4, -1.05, 0.0, 0.0])
    rng = np.random.default_rng(5)
    st[O.F_AT:O.F_AT + 6] += 1e-3 * rng.standard_normal((6,) + cfg.shape[1:])
    norms, H, M = O.constraints(cfg, st)
    X, Y, Z = _mesh(cfg)
    C = np.stack([_int(cfg, H)] + [_int(cfg, M[i]) for i in range(3)]).reshape(4, -1)
    keep = np.ones(C.shape[1], bool)
    for (m, px, py, pz) in cfg.punctures:
        r = np.sqrt((X - px) ** 2 + (Y - py) ** 2 + (Z - pz) ** 2)
        keep &= _int(cfg, r).reshape(-1) > cfg.r_excise
    np.testing.assert_allclose(norms[0:4], np.sqrt((C ** 2).mean(axis=1)), rtol=1e-12)
    np.testing.assert_allclose(norms[4:8], np.abs(C).max(axis=1), rtol=1e-15)
    np.testing.assert_allclose(norms[8:12], np.sqrt((C[:, keep] ** 2).mean(axis=1)), rtol=1e-12)
    np.testing.assert_allclose(norms[12:16], np.abs(C[:, keep]).max(axis=1), rtol=1e-15)
    assert keep.sum() < keep.size
