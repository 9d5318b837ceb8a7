"""Pins for the instrumented oracle build (oracle/bssn_oracle_instrumented.cpp):
the rounding scale that the float64 parity bars use, and the operation count.

The instrumented build evaluates the oracle's point-wise right-hand side
(Sec. "Spacetime Curvature Evolution", with the Sommerfeld boundary of Sec.
"Boundary Conditions" on ghost points) from the same header as the plain
oracle, carrying beside each float64 value the magnitude M of the same
expression evaluated on absolute values.  For sums of products the rounding
error of any evaluation order is bounded by gamma_n M (Higham, Sec. 3.3), so
two float64 evaluations of the same right-hand side in different orders -- the
oracle's printed arrangement and the GPU's rearranged one -- differ by a small
multiple of u M, u = 2^-53.

Pinned here, against things other than the instrumented build itself:
* its values equal the plain oracle's bit for bit (same operations, same order);
* M >= |value| (a sum of absolute values bounds the absolute value of the sum);
* an evaluation of the same header in long double (far smaller unit roundoff)
  lies within a few u M of the float64 one at every point and field, interior
  and ghost, in both conformal variants and with matter sources;
* a planted extra rounding (the state perturbed by one ulp-scale relative
  change of 1e-13) moves the right-hand side by far more than u M at some
  point, so the bar is not vacuous."""
import numpy as np
import pytest

import oracle as O
from paper_1111_3344_gb300 import inputs

U = 2.0 ** -53


def _case(use_w, matter=False, shift="gamma-driver"):
    n = (13, 11, 12)
    xmin = (-2.1, -1.7, -1.9)
    h = 0.33
    tm = inputs.random_tmunu(3, n, xmin, h) if matter else None
    cfg = O.Config(n=n, xmin=xmin, h=h, periodic=False, use_w=use_w, shift=shift,
                   punctures=[(0.7, 0.11, -0.05, 0.08)], tmunu=tm)
    bg = O.initial_data(cfg, "bl", [1, 0.7, 0.11, -0.05, 0.08])
    st = inputs.random_state(5, n, xmin, h, amp=0.05, background=bg)
    ext = [n[d] + 6 for d in range(3)]
    ijk = np.array([(i, j, k) for i in range(0, ext[0], 2) for j in range(0, ext[1], 2)
                    for k in range(0, ext[2], 2)], dtype=np.int32)
    return cfg, st, ijk


@pytest.mark.parametrize("use_w", [True, False])
@pytest.mark.parametrize("matter", [False, True])
def test_magnitude_bounds_rounding_error(use_w, matter):
    cfg, st, ijk = _case(use_w, matter)
    val, mag = O.rhs_points_mag(cfg, st, ijk)
    assert np.array_equal(val, O.rhs_points(cfg, st, ijk))
    assert (mag >= np.abs(val)).all()
    ext = O.rhs_points_ext(cfg, st, ijk)
    # the float64 evaluation against the extended one: measured 1.3 u M at
    # worst; the first-order bound gamma_n M has n in the hundreds
    ratio = np.abs(val - ext) / mag
    assert ratio.max() <= 16 * U, ratio.max() / U
    # the extended evaluation really differs from the float64 one (it is not
    # the same computation), and the bar is far tighter than the values
    assert (val != ext).any()
    assert np.median(mag) < 1e4 * np.median(np.abs(val))


def test_magnitude_bar_is_not_vacuous():
    """A relative change of 1e-13 in the state (about 450 u) changes the
    right-hand side by more than 16 u M somewhere: a bar of that size sees
    errors of the state's own rounding scale."""
    cfg, st, ijk = _case(True)
    val, mag = O.rhs_points_mag(cfg, st, ijk)
    rng = np.random.default_rng(0)
    st2 = st * (1.0 + 1e-13 * rng.standard_normal(st.shape))
    val2 = O.rhs_points(cfg, st2, ijk)
    assert (np.abs(val2 - val) / mag).max() > 16 * U


@pytest.mark.parametrize("use_w", [True, False])
def test_operation_count(use_w):
    """The count of the printed arrangement at an interior point: the same at
    every interior point (the arrangement has no data-dependent work), fewer
    with a frozen shift (no beta and B equations, no advection of them), and
    more on a ghost point (the interior point it recurses to, plus the
    boundary terms)."""
    cfg, st, _ = _case(use_w)
    a = O.rhs_opcount(cfg, st, (8, 7, 8))
    b = O.rhs_opcount(cfg, st, (4, 12, 5))
    assert a == b
    flops = a["add"] + a["mul"] + a["div"]
    assert 5000 < flops < 50000
    cfg_f, st_f, _ = _case(use_w, shift="frozen")
    fr = O.rhs_opcount(cfg_f, st_f, (8, 7, 8))
    assert fr["add"] + fr["mul"] + fr["div"] < flops
    gh = O.rhs_opcount(cfg, st, (1, 7, 8))
    assert gh["add"] + gh["mul"] + gh["div"] > flops
