"""Parity of the analysis steps after the evolution (through the C ABI) with
the oracle: the ADM mass / angular momentum volume integrals (Sec. "Masses
and Momenta") and the puncture tracker (Sec. "Object tracking").

Bars (float64):
* integrands: per component, error <= 1e-12 of the component's largest
  magnitude; the mass integrand, a difference of far larger terms (the
  conformal Ricci scalar sums 81 second differences), also gets the rounding
  scale of those terms (see _m_rounding);
* integrals: |gpu - oracle| <= h^3 (N 1e-12 max|integrand| + 1e-13 sum
  |integrand|) over the N interior points: the pointwise bound summed, plus
  the rounding of two summation orders;
* tracked positions: 1e-12 relative to the largest position coordinate per
  step (one interpolation of the shift and one multiply-add).
Inputs come from the oracle, exact solutions or the seeded generators, never
from the CUDA path."""
import numpy as np
import pytest

import exact_solutions as E
import oracle as O
from cases import bl_params, gpu_params, normwise_errors, oracle_cfg
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


def _m_rounding(st, h, use_w):
    """Rounding scale of the mass integrand: it is a difference of terms far
    larger than itself, e^{5 phi}(At.At - 2K^2/3) and e^{phi} Rt, and Rt sums
    81 second differences of gt_ij, each rounding by up to 64 eps max|gt| /
    (12 h^2).  Two evaluations in different orders differ by at most twice
    the sum, with a factor 10 margin."""
    inner = (slice(3, -3),) * 3
    chi = st[O.F_CHI][inner]
    psi = np.maximum(chi, 1e-10) ** -0.5 if use_w else np.exp(chi)
    gmax = np.abs(st[O.F_GT:O.F_GT + 6][(slice(None),) + inner]).max()
    amax = np.abs(st[O.F_AT:O.F_AT + 6][(slice(None),) + inner]).max()
    kmax = np.abs(st[O.F_TRK][inner]).max()
    eps = np.finfo(np.float64).eps
    rt = 10 * 2 * 81 * 64 * eps * gmax / (12 * h * h) * psi.max()
    kk = 10 * 2 * 50 * eps * (psi ** 5).max() * (9 * amax * amax * gmax ** 2 + kmax * kmax)
    return (rt + kk) / (16 * np.pi)


def _check_integrals(got_i, got_d, want_i, want_d, h, m_round):
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    flat = np.abs(want_d[inner]).reshape(4, -1)
    # pointwise: 1e-12 of each integrand's largest magnitude, floored at 1e-3
    # of the largest of the four (as in normwise_errors: an integrand that
    # vanishes identically still carries rounding of the others' size); the
    # mass integrand also gets its rounding scale (a cancellation of larger
    # terms)
    scale = np.maximum(flat.max(axis=1), 1e-3 * flat.max())
    tol = 1e-12 * scale + np.array([m_round, 0.0, 0.0, 0.0])
    err = np.abs(got_d[inner] - want_d[inner]).reshape(4, -1).max(axis=1)
    assert (err <= tol).all(), (err, tol, normwise_errors(got_d[inner], want_d[inner]))
    # integrals: the sum of the pointwise bounds plus the rounding of two
    # summation orders
    mag = (tol * flat.shape[1] + 1e-13 * flat.sum(axis=1)) * h ** 3
    bound = np.concatenate([mag, mag]) + 1e-300
    assert (np.abs(got_i - want_i) <= bound).all(), (got_i, want_i, bound)


@pytest.mark.parametrize("name,box,periodic", [("ks_wavy", (1.5, 2.5), False), ("flat_wavy", (-0.5, 0.5), False),
                                               ("gauge_wave", (-0.5, 0.5), True)])
@pytest.mark.parametrize("conformal", ["W", "phi"])
def test_adm_integrals_exact_spacetimes(torch_cuda, name, box, periodic, conformal):
    lo, hi = box
    case = dict(n=(21, 18, 23), xmin=(lo, lo, lo), h=(hi - lo) / 21,
                boundary="periodic" if periodic else "sommerfeld", conformal=conformal,
                punctures=[(1.0, lo + 0.4, lo + 0.5, lo + 0.6)], r_excise=0.3)
    cfg = oracle_cfg(case)
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    st, _, _ = E.evaluate(name, Xc, Yc, Zc, use_w=conformal == "W")
    want_i, want_d = O.adm_integrals(cfg, st)
    evo = _evo(case)
    evo.set_state(st, 0.0)
    evo.set_punctures(case["punctures"])
    got_i, got_d = evo.adm_integrals(densities=True)
    _check_integrals(got_i, got_d, want_i, want_d, case["h"], _m_rounding(st, case["h"], conformal == "W"))
    assert got_i[0] != got_i[4]  # the excised set is a proper subset here
    evo.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adm_integrals_perturbed_bl(torch_cuda, precision):
    """A perturbed two-puncture state: every term of both integrands is live;
    the integrals are float64 in every precision mode."""
    case = dict(n=(34, 20, 17), xmin=(-3.0, -2.0, -1.5), h=0.18, boundary="sommerfeld", conformal="W",
                punctures=[(0.6, 0.71, 0.02, 0.01), (0.4, -0.93, -0.05, 0.03)], r_excise=0.5,
                precision=precision)
    cfg = oracle_cfg(case)
    bg = O.initial_data(cfg, "bl", bl_params(case))
    st = inputs.random_state(21, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    want_i, want_d = O.adm_integrals(cfg, st)
    evo = _evo(case)
    evo.set_initial_data("bl", bl_params(case))  # sets the punctures
    evo.set_state(st, 0.0)
    got_i, got_d = evo.adm_integrals(densities=True)
    _check_integrals(got_i, got_d, want_i, want_d, case["h"], _m_rounding(st, case["h"], True))
    got_i2, _ = evo.adm_integrals(densities=False)
    assert np.array_equal(got_i, got_i2)  # deterministic reduction
    evo.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tracker_follows_oracle(torch_cuda, precision):
    """Punctures (inside, next to the block edge and in the ghost zone) moved
    by the GPU during RK4 steps against oracle Euler steps on the GPU's own
    y_n at the start of each step."""
    case = dict(n=(30, 22, 18), xmin=(-2.5, -2.0, -1.5), h=0.17, boundary="sommerfeld", conformal="W",
                punctures=[(0.6, 0.51, 0.03, -0.02), (0.4, -0.87, -0.11, 0.05)], r_excise=0.4,
                precision=precision)
    cfg = oracle_cfg(case)
    bg = O.initial_data(cfg, "bl", bl_params(case))
    st = inputs.random_state(5, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    # a shift of order 0.3 so that the punctures move measurably
    st[O.F_BETA:O.F_BETA + 3] += np.array([0.3, -0.2, 0.25])[:, None, None, None]
    pts = [(0.6, 0.51, 0.03, -0.02), (0.4, -0.87, -0.11, 0.05), (0.1, 2.41, 1.69, 1.3),
           (0.1, -2.9, -2.45, -1.95)]
    evo = _evo(case)
    evo.set_state(st, 0.0)
    evo.set_punctures(pts)
    evo.track_punctures(True)
    want = np.array(pts, dtype=np.float64)
    for _ in range(3):
        y_n, _ = evo.get_state()
        want = O.track_step(cfg, y_n, want, cfg.dt)
        evo.rk4_step(1)
        got = evo.get_punctures()
        assert got.shape == want.shape
        assert np.abs(got[:, 0] - want[:, 0]).max() == 0.0
        err = np.abs(got[:, 1:] - want[:, 1:]).max()
        assert err <= 1e-12 * np.abs(want[:, 1:]).max(), (got, want)
    assert np.abs(want[:, 1:] - np.array(pts)[:, 1:]).min() > 1e-3  # they moved
    # the excised constraint norms follow the tracked positions
    y_n, _ = evo.get_state()
    cfg.punctures = [tuple(r) for r in evo.get_punctures()]
    norms_want, _, _ = O.constraints(cfg, y_n)
    norms_got = evo.constraints()
    np.testing.assert_allclose(norms_got, norms_want, rtol=1e-11, atol=1e-300)
    # tracking off: positions stay
    evo.track_punctures(False)
    before = evo.get_punctures()
    evo.rk4_step(1)
    assert np.array_equal(evo.get_punctures(), before)
    evo.close()


def test_tracker_zero_shift_and_no_punctures(torch_cuda):
    case = dict(n=(12, 12, 12), xmin=(-1.0, -1.0, -1.0), h=1.0 / 6, boundary="sommerfeld", conformal="W")
    evo = _evo(case)
    evo.set_initial_data("flat", [])
    evo.track_punctures(True)
    evo.rk4_step(2)  # no punctures: nothing to move
    assert evo.get_punctures().shape == (0, 4)
    evo.set_punctures([(1.0, 0.1, 0.2, 0.3)])
    evo.rk4_step(2)  # flat space: beta = 0, the puncture stays exactly
    np.testing.assert_array_equal(evo.get_punctures(), [[1.0, 0.1, 0.2, 0.3]])
    evo.close()


def _psi4_rounding(st, h, use_w):
    """Rounding scale of Psi4: the Ricci tensor contracted with the triad sums
    about 400 second differences of gamma_ij (each rounding by up to
    64 eps max|gamma| / (12 h^2)), the Codazzi term about 100 first
    differences of K_ij (18 eps max|K| / (12 h)) and the K K terms about 50
    products; two evaluations in different orders differ by at most twice
    the sum, with a factor 10 margin."""
    inner = (slice(3, -3),) * 3
    chi = st[O.F_CHI][inner]
    e4 = np.maximum(chi, 1e-10) ** -2 if use_w else np.exp(4 * chi)
    gmax = np.abs(st[O.F_GT:O.F_GT + 6][(slice(None),) + inner]).max() * e4.max()
    kmax = (np.abs(st[O.F_AT:O.F_AT + 6][(slice(None),) + inner]).max()
            + np.abs(st[O.F_TRK][inner]).max()) * e4.max()
    eps = np.finfo(np.float64).eps
    return 10 * 2 * eps * (400 * 64 * gmax / (12 * h * h) + 100 * 18 * kmax / (12 * h) + 50 * kmax * kmax)


def _check_psi4(got, want, st, h, use_w):
    inner = (slice(None), slice(3, -3), slice(3, -3), slice(3, -3))
    err = np.abs(got[inner] - want[inner]).max()
    tol = 1e-12 * np.abs(want[inner]).max() + _psi4_rounding(st, h, use_w)
    assert err <= tol, (err, tol, np.abs(want[inner]).max())
    return err


@pytest.mark.parametrize("name,box,periodic", [("ks_wavy", (1.5, 2.5), False), ("ks_offset", (1.5, 2.5), False),
                                               ("ks_boost", (1.5, 2.5), False), ("flat_wavy", (-0.5, 0.5), False),
                                               ("gauge_wave", (-0.5, 0.5), True)])
@pytest.mark.parametrize("conformal", ["W", "phi"])
def test_psi4_exact_spacetimes(torch_cuda, name, box, periodic, conformal):
    lo, hi = box
    case = dict(n=(21, 18, 23), xmin=(lo, lo, lo), h=(hi - lo) / 21,
                boundary="periodic" if periodic else "sommerfeld", conformal=conformal)
    cfg = oracle_cfg(case)
    Zc, Yc, Xc = np.meshgrid(cfg.coords(2), cfg.coords(1), cfg.coords(0), indexing="ij")
    st, _, _ = E.evaluate(name, Xc, Yc, Zc, use_w=conformal == "W")
    want = O.psi4(cfg, st)
    evo = _evo(case)
    evo.set_state(st, 0.0)
    got = evo.psi4_to_numpy(evo.psi4())
    err = _check_psi4(got, want, st, case["h"], conformal == "W")
    print(f"psi4 {name} {conformal}: max |gpu - oracle| = {err:.3e}, max |psi4| = {np.abs(want).max():.3e}")
    evo.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_psi4_perturbed_bl_and_axis(torch_cuda, precision):
    """A perturbed two-puncture state on a grid with cell centres on the z
    axis (x = y = 0), where Psi4 is 0 by definition."""
    h = 0.18
    case = dict(n=(33, 21, 17), xmin=(-16.5 * h, -10.5 * h, -1.5), h=h, boundary="sommerfeld", conformal="W",
                punctures=[(0.6, 0.71, 0.02, 0.01), (0.4, -0.93, -0.05, 0.03)], precision=precision)
    cfg = oracle_cfg(case)
    bg = O.initial_data(cfg, "bl", bl_params(case))
    st = inputs.random_state(23, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    want = O.psi4(cfg, st)
    evo = _evo(case)
    evo.set_state(st, 0.0)
    got = evo.psi4_to_numpy(evo.psi4())
    err = _check_psi4(got, want, st, case["h"], True)
    print(f"psi4 perturbed BL ({precision}): max |gpu - oracle| = {err:.3e}, max |psi4| = {np.abs(want).max():.3e}")
    X = cfg.coords(0)
    Y = cfg.coords(1)
    i0, j0 = int(np.argmin(np.abs(X))), int(np.argmin(np.abs(Y)))
    assert X[i0] == 0.0 and Y[j0] == 0.0
    assert np.all(got[:, 3:-3, j0, i0] == 0.0)
    assert np.abs(got[:, 3:-3, j0, i0 + 1]).min() > 0.0
    evo.close()
