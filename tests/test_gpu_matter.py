"""Parity of the matter-coupled path (through the C ABI) with the oracle:
right-hand side, RK4 steps, constraint norms and ADM integrals with a
stress-energy tensor T_{mu nu} (Sec. "Spacetime Curvature Evolution" source
terms, Sec. "TmunuBase").

Inputs: the exact dust FLRW universe in tilted coordinates (T_{mu nu} exact)
and a perturbed Brill-Lindquist state with a seeded smooth T_{mu nu}
(paper_1111_3344_gb300.inputs.random_tmunu).  Bars as for vacuum: float64
right-hand side 1e-12 normwise per field (for the sourced fields of the
exact data, whose exact right-hand side is a cancellation, 1e-12 of the
oracle's magnitude of the terms where that is larger), RK4 steps 1e-11; constraint norms and ADM integrands to the rounding scale of the
terms that cancel in them; mixed right-hand side 1e-4 normwise (the float32
bar of the vacuum mixed tests)."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O
from cases import bl_params, gpu_params, normwise_errors, oracle_cfg, rounding_aware_errors
from paper_1111_3344_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


def _evo(case):
    from paper_1111_3344_gb300.bssn import Evolution
    return Evolution(gpu_params(case))


FLRW = dict(n=(20, 17, 23), xmin=(-0.5, -0.45, -0.6), h=0.05, boundary="sommerfeld", conformal="W")
BLM = dict(n=(30, 19, 17), xmin=(-2.7, -1.7, -1.5), h=0.18, boundary="sommerfeld", conformal="W",
           punctures=[(0.6, 0.51, 0.03, -0.02), (0.4, -0.87, -0.11, 0.05)], r_excise=0.4)


def _flrw(case):
    cfg = oracle_cfg(case)
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    st, _, grad = E.evaluate("flrw_dust", Xc, Yc, Zc, use_w=case["conformal"] == "W")
    return cfg, st, np.ascontiguousarray(grad["tmunu"])


def _blm(case, seed=31):
    cfg = oracle_cfg(case)
    bg = O.initial_data(cfg, "bl", bl_params(case))
    st = inputs.random_state(seed, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    tm = inputs.random_tmunu(seed + 1, case["n"], case["xmin"], case["h"], amp=0.02)
    return cfg, st, tm


@pytest.mark.parametrize("which", ["flrw", "bl"])
@pytest.mark.parametrize("conformal", ["W", "phi"])
def test_rhs_with_matter(torch_cuda, which, conformal):
    case = dict(FLRW if which == "flrw" else BLM, conformal=conformal)
    cfg, st, tm = _flrw(case) if which == "flrw" else _blm(case)
    cfg.tmunu = tm
    want, mag = O.rhs_mag(cfg, st)
    evo = _evo(case)
    evo.set_matter(tm)
    got = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    e = normwise_errors(got, want)
    if which == "bl":
        assert e.max() <= 1e-12, dict(zip(O.FIELD_NAMES, e))
    else:
        # Exact data: the exact d_t of K, At, Gt^i, B^i is a small difference of
        # its curvature, gauge and matter terms (Gt^z: 0.05 against terms of
        # 0.4), so two float64 evaluations in different orders differ by a few
        # ulps of those terms: the bar is 1e-12 of the larger of the field's
        # scale and the oracle's magnitude of the terms at the point
        # (cases.rounding_aware_errors); fields without a source term keep the
        # plain normwise 1e-12.
        r = rounding_aware_errors(got, want, mag)
        assert r.max() <= 1.0, (dict(zip(O.FIELD_NAMES, r)), dict(zip(O.FIELD_NAMES, e)))
        src = [O.F_TRK] + list(range(O.F_AT, O.F_AT + 6)) + list(range(O.F_GAM, O.F_GAM + 3)) + \
            list(range(O.F_B, O.F_B + 3))
        rest = [f for f in range(O.NF) if f not in src]
        assert e[rest].max() <= 1e-12, dict(zip(O.FIELD_NAMES, e))
    # the matter changes K, At, Gt and B: vacuum differs there
    evo.set_matter(None)
    vac = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    cfg.tmunu = None
    np.testing.assert_allclose(vac, O.rhs(cfg, st), rtol=0, atol=1e-12 * np.abs(want).max())
    assert np.abs(vac[O.F_TRK] - got[O.F_TRK]).max() > 1e-3
    evo.close()


def test_rk4_with_matter(torch_cuda):
    case = dict(BLM)
    cfg, st, tm = _blm(case)
    cfg.tmunu = tm
    want = O.rk4(cfg, st, 3)
    evo = _evo(case)
    evo.set_matter(tm)
    evo.set_state(st, 0.0)
    evo.rk4_step(3)
    got, _ = evo.get_state()
    e = normwise_errors(got, want)
    assert e.max() <= 1e-11, dict(zip(O.FIELD_NAMES, e))
    evo.close()


def test_mixed_rhs_with_matter(torch_cuda):
    case = dict(BLM, precision="mixed", w_fp64_threshold=0.2)
    cfg, st, tm = _blm(case)
    cfg.tmunu = tm
    want = O.rhs(cfg, st)
    evo = _evo(case)
    evo.set_matter(tm)
    got = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    e = normwise_errors(got, want)
    print("mixed matter rhs normwise errors", dict(zip(O.FIELD_NAMES, np.round(e, 9))))
    assert e.max() <= 1e-4, dict(zip(O.FIELD_NAMES, e))
    evo.close()


def test_constraints_and_integrals_with_matter(torch_cuda):
    case = dict(FLRW, punctures=[(1.0, 0.1, 0.0, 0.0)], r_excise=0.2)
    cfg, st, tm = _flrw(case)
    cfg.tmunu = tm
    norms_want, _, _ = O.constraints(cfg, st)
    ints_want, dens_want = O.adm_integrals(cfg, st)
    evo = _evo(case)
    evo.set_state(st, 0.0)
    evo.set_punctures(case["punctures"])
    evo.set_matter(tm)
    # H (about 1e-4 here, the truncation error) is a difference of O(1) terms:
    # R (about 100 second differences of gamma_ij, each rounding by up to
    # 64 eps max|gamma| / (12 h^2)), K^2 - K.K and 16 pi E; M_i likewise with
    # first differences of K_ij.  The norms agree to that rounding scale.
    eps = np.finfo(np.float64).eps
    h = case["h"]
    gmax = np.abs(st[O.F_GT:O.F_GT + 6]).max() / np.min(st[O.F_CHI]) ** 2
    kmax = (np.abs(st[O.F_AT:O.F_AT + 6]).max() + np.abs(st[O.F_TRK]).max()) / np.min(st[O.F_CHI]) ** 2
    atol_h = 100 * 64 * eps * gmax / (12 * h * h)
    atol_m = 100 * 18 * eps * kmax / (12 * h)
    atol = np.array(([atol_h] + [atol_m] * 3) * 4)
    got_n = evo.constraints()
    assert (np.abs(got_n - norms_want) <= 1e-12 * np.abs(norms_want) + atol).all(), (got_n, norms_want, atol)
    ints, dens = evo.adm_integrals(densities=True)
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    # the mass integrand is the same kind of cancellation (R-tilde, 16 pi E,
    # 2K^2/3), times e^{5 phi} / (16 pi)
    psi5 = np.min(st[O.F_CHI]) ** -2.5  # e^{5 phi} = W^{-5/2}
    tol_d = 1e-12 * np.abs(dens_want[inner]).reshape(4, -1).max(axis=1) + \
        np.array([psi5 * (81 * 64 * eps * gmax / (12 * h * h)) * 10 / (16 * np.pi), 0.0, 0.0, 0.0])
    err_d = np.abs(dens[inner] - dens_want[inner]).reshape(4, -1).max(axis=1)
    assert (err_d <= tol_d + 1e-300).all(), (err_d, tol_d)
    npts = np.prod(case["n"])
    tol_i = np.concatenate([tol_d, tol_d]) * npts * h ** 3 + 1e-13 * np.abs(ints_want)
    assert (np.abs(ints - ints_want) <= tol_i).all(), (ints, ints_want, tol_i)
    # the sources matter: vacuum norms are far larger (16 pi E is O(1) here)
    evo.set_matter(None)
    assert evo.constraints()[0] > 100 * norms_want[0]
    evo.close()
