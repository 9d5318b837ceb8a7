"""Pins for the oracle's RK4 method of lines and the algebraic (non-derivative)
terms of the BSSN equations: the Kasner spacetime of the paper's Sec.
"Cosmology" (initial data gamma = delta, K_ij = diag(-2/3, -2/3, 1/3) at t = 1,
alpha = 1, beta = 0), evolved with the time-step sequence of the Kasner
figure (dt = 0.1, 0.05, 0.025, 0.0125); errors against the closed form fall
16x per halving of dt (fourth order).

The data are homogeneous, so every spatial derivative vanishes and the
evolution is an ODE in proper time tau with d tau = alpha dt:
  W = tau^{-1/3} (phi = ln(tau)/6), gt = diag(tau^{2/3}, tau^{2/3}, tau^{-4/3}),
  K = -1/tau, At = diag(-tau^{-1/3}/3, -tau^{-1/3}/3, 2 tau^{-7/3}/3).
Slicing fixes tau(t): geodesic (alpha = 1) tau = t; harmonic (d_t alpha =
-alpha^2 K = alpha^2/tau) alpha = tau, tau = e^{t-1}; 1+log (d_t alpha =
-2 alpha K) alpha = 1 + 2 ln tau, t - 1 = int_1^tau ds / (1 + 2 ln s)."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle as O


def kasner_state(cfg, tau, alpha):
    st = np.zeros(cfg.shape)
    st[O.F_CHI] = tau ** (-1 / 3) if cfg.use_w else math.log(tau) / 6
    st[O.F_GT + 0] = st[O.F_GT + 3] = tau ** (2 / 3)
    st[O.F_GT + 5] = tau ** (-4 / 3)
    st[O.F_TRK] = -1.0 / tau
    st[O.F_AT + 0] = st[O.F_AT + 3] = -tau ** (-1 / 3) / 3
    st[O.F_AT + 5] = 2 * tau ** (-7 / 3) / 3
    st[O.F_ALP] = alpha
    return st


def tau_alpha(slicing, t):
    if slicing == "geodesic":
        return t, 1.0
    if slicing == "harmonic":
        tau = math.exp(t - 1.0)
        return tau, tau
    f = lambda tau: integrate.quad(lambda s: 1.0 / (1.0 + 2.0 * math.log(s)), 1.0, tau,  # noqa: E731
                                   epsabs=1e-15, epsrel=1e-14)[0] - (t - 1.0)
    tau = optimize.brentq(f, 1.0, 10.0, xtol=1e-15, rtol=1e-15)
    return tau, 1.0 + 2.0 * math.log(tau)


@pytest.mark.parametrize("use_w", [True, False])
def test_kasner_initial_data_matches_closed_form(use_w):
    cfg = O.Config(n=(4, 4, 4), h=0.25, periodic=True, use_w=use_w)
    st = O.initial_data(cfg, "kasner", [1.0])
    np.testing.assert_allclose(st, kasner_state(cfg, 1.0, 1.0), atol=1e-15)
    st2 = O.initial_data(cfg, "kasner", [1.7])
    np.testing.assert_allclose(st2, kasner_state(cfg, 1.7, 1.0), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("slicing", ["geodesic", "harmonic", "1+log"])
@pytest.mark.parametrize("use_w", [True, False])
def test_kasner_rk4_fourth_order(slicing, use_w):
    t_end = 2.0
    errs = []
    for dt in (0.1, 0.05, 0.025, 0.0125):
        cfg = O.Config(n=(4, 4, 4), h=0.25, periodic=True, use_w=use_w, slicing=slicing,
                       shift="gamma-driver", eta=2.0, dt=dt, ko_eps=0.1)
        st = O.initial_data(cfg, "kasner", [1.0])
        nsteps = int(round((t_end - 1.0) / dt))
        out = O.rk4(cfg, st, nsteps)
        tau, alpha = tau_alpha(slicing, t_end)
        exact = kasner_state(cfg, tau, alpha)
        errs.append(np.abs(out - exact).max(axis=(1, 2, 3)))
        # homogeneity is preserved exactly; the shift stays zero up to the
        # rounding of stencil sums over equal values
        assert np.all(out == out[:, :1, :1, :1])
        assert np.abs(out[O.F_BETA:]).max() < 1e-14
    errs = np.array(errs)
    moving = [O.F_CHI, O.F_GT, O.F_GT + 3, O.F_GT + 5, O.F_TRK, O.F_AT, O.F_AT + 3, O.F_AT + 5]
    if slicing != "geodesic":
        moving.append(O.F_ALP)
    for f in moving:
        r = errs[:-1, f] / errs[1:, f]
        # fourth order: ratios approach 2^4 = 16 as dt -> 0
        assert np.all((r > 12.0) & (r < 22.0)), (O.FIELD_NAMES[f], errs[:, f], r)
        assert 14.5 < r[-1] < 17.5, (O.FIELD_NAMES[f], errs[:, f], r)
    assert errs[-1].max() < 1e-7
