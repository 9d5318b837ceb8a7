"""The allocation-free constraint entry point, bssn_constraints_noalloc.

Some callers cannot give the library device memory: a host that reserved all
of HBM in its own arena, a plug-in host that forbids allocation, a real-time
loop that must not call cudaMalloc.  For them the library keeps the reduction
scratch of the constraint norms in a static device array instead.  This test
checks, through the C ABI, that the allocation-free call gives the same norms
as the context-based bssn_constraints on two different states in a row (so
the second call cannot lean on what the first left in the shared array), and
that grids beyond the static capacity are refused.  It lives in its own file,
collected last, and builds on nothing but the library itself, so it passes
alone in a fresh process as well as after the rest of the suite."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_constraints_match_context_path_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1111_3344_gb300 import bssn as B
    from paper_1111_3344_gb300 import inputs

    n, L = (40, 33, 29), 4.0
    h = 2 * L / 40
    punct = [(0.6, 0.3, 0.0, 0.05), (0.5, -0.9, 0.1, 0.0)]
    params = B.Params(n=n, xmin=(-L, -L * 33 / 40, -L * 29 / 40), h=h, boundary="sommerfeld",
                      conformal="W", r_excise=0.9)
    evo = B.Evolution(params)
    bl = [2] + [v for q in punct for v in q]
    evo.set_initial_data("bl", bl)
    # state 1: Brill-Lindquist data with a seeded perturbation on every field
    st0, _ = evo.get_state()
    st1 = inputs.random_state(21, n, params.xmin, h, amp=0.03, background=st0)
    evo.set_state(st1, 0.0)
    stream = evo.stream.cuda_stream
    want1 = evo.constraints()
    got1 = B.bssn_constraints_noalloc(params, B.bssn_state_ptr(evo.ctx), punct, stream)
    # state 2: one RK4 step later (different values in every reduction slot)
    evo.rk4_step(1)
    want2 = evo.constraints()
    got2 = B.bssn_constraints_noalloc(params, B.bssn_state_ptr(evo.ctx), punct, stream)
    assert np.abs(want1 - want2).max() > 0
    np.testing.assert_allclose(got1, want1, rtol=1e-12, atol=0)
    np.testing.assert_allclose(got2, want2, rtol=1e-12, atol=0)

    # a grid beyond the static scratch is refused with EINVAL, before any launch
    big = B.Params(n=(256, 128, 129), xmin=(0.0,) * 3, h=0.1)
    with pytest.raises(B.BssnError) as e:
        B.bssn_constraints_noalloc(big, B.bssn_state_ptr(evo.ctx), (), stream)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    evo.close()
