"""Pins for the oracle's BSSN right-hand side against exact vacuum spacetimes
(equations of the paper's Sec. "Spacetime Curvature Evolution").

For an exact solution of the vacuum Einstein equations, the right-hand sides
of phi/W, gt_ij, K, At_ij and Gt^i evaluated on its data equal the exact time
derivatives up to the O(h^4) truncation error of the stencils, in any gauge.
The data here (tests/exact_solutions.py) are flat space and Schwarzschild in
generic, time-dependent coordinates, so every term of every equation is
non-zero and a dropped term, a wrong sign, index or transposed operand leaves
an O(1) residual instead of a 16x drop per halving of h.  The gauge equations
(1+log / harmonic / geodesic slicing, Gamma-driver with q(r)) are checked
against their definitions evaluated with the exact fields and gradients."""
import math

import numpy as np
import pytest

import exact_solutions as E
import oracle as O

BOXES = {"flat_wavy": (-0.5, 0.5), "ks_wavy": (1.5, 2.5)}


def _setup(name, n, use_w, **kw):
    lo, hi = BOXES[name]
    h = (hi - lo) / n
    cfg = O.Config(n=(n, n, n), h=h, xmin=(lo, lo, lo), periodic=True, use_w=use_w, **kw)
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    state, dts, grad = E.on_grid(name, (n, n, n), lo, hi, use_w=use_w)
    return cfg, state, dts, grad, (Xc, Yc, Zc)


def _int(cfg, a):
    g = O.GHOST
    return a[..., g:g + cfg.n[2], g:g + cfg.n[1], g:g + cfg.n[0]]


def _expected_gauge(cfg, state, grad, X):
    """Gauge right-hand sides from their defining equations with exact values."""
    alpha, trK = state[O.F_ALP], state[O.F_TRK]
    beta = state[O.F_BETA:O.F_BETA + 3]
    B = state[O.F_B:O.F_B + 3]
    adv = lambda g: sum(beta[j] * g[j] for j in range(3))  # noqa: E731
    exp = {}
    if cfg.slicing == "1+log":
        exp[O.F_ALP] = adv(grad["alpha"]) - 2.0 * alpha * trK
    elif cfg.slicing == "harmonic":
        exp[O.F_ALP] = adv(grad["alpha"]) - alpha ** 2 * trK
    else:
        exp[O.F_ALP] = adv(grad["alpha"])
    r = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2)
    q = np.ones_like(r) if math.isinf(cfg.q_R) else np.where(r <= cfg.q_R, 1.0, cfg.q_R / r)
    for i in range(3):
        if cfg.shift == "frozen":
            exp[O.F_BETA + i] = np.zeros_like(alpha)
            exp[O.F_B + i] = np.zeros_like(alpha)
            continue
        exp[O.F_BETA + i] = adv(grad["beta"][i]) + 0.75 * B[i]
        dGt_noadv = grad["dt_Gt"][i] - adv(grad["Gt"][i])
        exp[O.F_B + i] = adv(grad["B"][i]) + dGt_noadv - cfg.eta * q * B[i]
    return exp


def _errors(name, n, use_w, **kw):
    cfg, state, dts, grad, X = _setup(name, n, use_w, **kw)
    grad["dt_Gt"] = dts[O.F_GAM:O.F_GAM + 3]
    r = O.rhs(cfg, state)
    exp = dict((f, dts[f]) for f in range(17))
    exp.update(_expected_gauge(cfg, state, grad, X))
    err = np.array([np.abs(_int(cfg, r[f] - exp[f])).max() for f in range(O.NF)])
    scale = np.array([np.abs(_int(cfg, exp[f])).max() for f in range(O.NF)])
    return err, scale


@pytest.mark.parametrize("name", ["flat_wavy", "ks_wavy"])
@pytest.mark.parametrize("use_w", [True, False])
def test_rhs_converges_to_exact_time_derivative(name, use_w):
    kw = dict(slicing="1+log", shift="gamma-driver", eta=0.7, ko_eps=0.1)
    e1, s1 = _errors(name, 12, use_w, **kw)
    e2, s2 = _errors(name, 24, use_w, **kw)
    # every evolved field is exercised: the exact time derivative is not small
    assert (s1[:17] > 1e-4).all(), s1
    ratio = e1 / np.maximum(e2, 1e-300)
    for f in range(O.NF):
        assert e2[f] < 2e-4 * max(s2[f], 1.0), (O.FIELD_NAMES[f], e2[f], s2[f])
        assert ratio[f] > 12.0, (O.FIELD_NAMES[f], e1[f], e2[f], ratio[f])


@pytest.mark.parametrize("slicing", ["harmonic", "geodesic"])
def test_other_slicings_and_q_of_r(slicing):
    kw = dict(slicing=slicing, shift="gamma-driver", eta=1.3, q_R=2.9, ko_eps=0.05)
    e1, _ = _errors("ks_wavy", 12, True, **kw)
    e2, _ = _errors("ks_wavy", 24, True, **kw)
    assert (e1 / e2 > 12.0).all(), e1 / e2


def test_frozen_shift_gauge_rhs_is_zero():
    kw = dict(slicing="1+log", shift="frozen", ko_eps=0.1)
    cfg, state, dts, grad, X = _setup("flat_wavy", 12, True, **kw)
    r = O.rhs(cfg, state)
    assert np.all(r[O.F_BETA:] == 0.0)


def test_gauge_wave_is_harmonic_with_zero_shift():
    """The gauge wave obeys harmonic slicing: the full right-hand side of all
    24 fields, lapse included, converges to the exact d_t."""
    errs = []
    for n in (12, 24):
        cfg = O.Config(n=(n, n, n), h=1.0 / n, xmin=(-0.5,) * 3, periodic=True,
                       slicing="harmonic", shift="frozen", ko_eps=0.1)
        Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
        state, dts, grad = E.evaluate("gauge_wave", Xc, Yc, Zc)
        dts[O.F_ALP] = grad["dt_alpha"]
        dts[O.F_BETA:] = 0.0
        r = O.rhs(cfg, state)
        errs.append(np.array([np.abs(_int(cfg, r[f] - dts[f])).max() for f in range(O.NF)]))
    big = errs[0] > 1e-12
    assert big[[0, 1, 4, 6, 7, 8, 11, 13, 14, 17]].all()
    assert (errs[0][big] / errs[1][big] > 12.0).all(), errs[0] / errs[1]
    assert (errs[1][~big] < 1e-11).all()
