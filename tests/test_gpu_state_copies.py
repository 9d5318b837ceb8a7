"""Asynchronous host copies of the state (bssn_set_state_async,
bssn_get_state_async, bssn_wait_state) against the synchronous ones.

The bar is bit equality, with and without device staging areas bound.
* A loop that uploads a state, steps and reads the state back every step
  gives the same host arrays through the asynchronous calls (read-back of
  step n overlapping the upload of step n+1) as through the synchronous ones.
* A read-back in the middle of an evolution does not change it: the mixed
  path reads back through its float shadow of y_n, which the next step must
  rebuild to the same bits."""
import numpy as np
import pytest

from cases import bl_params, gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


def _case(precision):
    # x extent a multiple of 32 (full-row kernels) and ragged y, z tiles
    return dict(n=(32, 22, 18), xmin=(-4.0, -2.75, -2.25), h=0.25, boundary="sommerfeld", conformal="W",
                slicing="1+log", shift="gamma-driver", eta=2.0, punctures=[(1.0, 0.05, 0.0, 0.0)],
                precision=precision, w_fp64_threshold=0.3)


def _pinned(torch, shape):
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


@pytest.mark.parametrize("staging", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pipelined_copies_match_synchronous(torch_cuda, precision, staging):
    """With device staging areas bound (bssn_set_staging), the uploads run on
    their own stream while the previous step may still be running."""
    from paper_1111_3344_gb300 import bssn as B
    c = _case(precision)
    evo = B.Evolution(gpu_params(c))
    evo.set_initial_data("bl", bl_params(c))
    evo.rk4_step(2)
    st0, _ = evo.get_state()
    steps = 3
    want = []
    for s in range(steps):
        evo.set_state(st0 * (1.0 + 1e-3 * s), 0.5 * s)
        evo.rk4_step(1)
        want.append(evo.get_state())
    if staging:
        evo.enable_copy_staging()
    host_in = [_pinned(torch_cuda, evo.shape) for _ in range(steps)]
    host_out = [_pinned(torch_cuda, evo.shape) for _ in range(steps)]
    times = []
    for s in range(steps):
        host_in[s][...] = st0 * (1.0 + 1e-3 * s)
        B.bssn_set_state_async(evo.ctx, host_in[s], 0.5 * s)
        evo.rk4_step(1)
        times.append(B.bssn_get_state_async(evo.ctx, host_out[s]))
    B.bssn_wait_state(evo.ctx)
    for s in range(steps):
        assert np.array_equal(host_out[s], want[s][0]), s
        assert times[s] == want[s][1]
    evo.close()


@pytest.mark.parametrize("staging", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_read_back_mid_evolution_leaves_it_unchanged(torch_cuda, precision, staging):
    from paper_1111_3344_gb300 import bssn as B
    c = _case(precision)
    a = B.Evolution(gpu_params(c))
    b = B.Evolution(gpu_params(c))
    if staging:
        a.enable_copy_staging()
    for e in (a, b):
        e.set_initial_data("bl", bl_params(c))
    a.rk4_step(2)
    mid = _pinned(torch_cuda, a.shape)
    B.bssn_get_state_async(a.ctx, mid)
    a.rk4_step(2)
    B.bssn_wait_state(a.ctx)
    b.rk4_step(2)
    want_mid, _ = b.get_state()
    b.rk4_step(2)
    assert np.array_equal(mid, want_mid)
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    a.close()
    b.close()


def test_staging_rejects_small_or_misaligned_blocks(torch_cuda):
    from paper_1111_3344_gb300 import bssn as B
    c = _case("fp64")
    evo = B.Evolution(gpu_params(c))
    p = evo.params.c()
    n = int(B.load().bssn_staging_bytes(B.ctypes.byref(p)))
    assert n >= 2 * 24 * int(np.prod(evo.shape[1:])) * 8
    buf = torch_cuda.empty(n + 256, dtype=torch_cuda.uint8, device="cuda")
    base = buf.data_ptr()
    assert B.load().bssn_set_staging(B.ctypes.c_void_p(evo.ctx), B.ctypes.c_void_p(base), n - 8) == 2  # ENOMEM
    assert B.load().bssn_set_staging(B.ctypes.c_void_p(evo.ctx), B.ctypes.c_void_p(base + 8), n) == 1  # EINVAL
    assert B.load().bssn_set_staging(B.ctypes.c_void_p(evo.ctx), B.ctypes.c_void_p(base), n) == 0
    assert B.load().bssn_set_staging(B.ctypes.c_void_p(evo.ctx), None, 0) == 0
    evo.close()


def test_upload_shadow_matches_shadow_kernel(torch_cuda):
    """Mixed path: an upload forms the float shadow of y_n inside its repack;
    the step after it equals, bit for bit, the step of an evolution whose
    shadow comes from the separate shadow kernel (after initial data)."""
    from paper_1111_3344_gb300 import bssn as B
    c = _case("mixed")
    a = B.Evolution(gpu_params(c))
    b = B.Evolution(gpu_params(c))
    a.set_initial_data("bl", bl_params(c))
    st, _ = a.get_state()
    b.set_state(st, 0.0)
    a.rk4_step(2)
    b.rk4_step(2)
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    a.close()
    b.close()


@pytest.mark.parametrize("staging", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_periodic_uploads(torch_cuda, precision, staging):
    """Periodic grids: the step after an upload refreshes the ghosts of y_n and
    (mixed) forms the float shadow from them; the asynchronous loop equals the
    synchronous one, and a state uploaded with inconsistent ghosts evolves as
    the same state with its ghosts filled."""
    from paper_1111_3344_gb300 import bssn as B
    from paper_1111_3344_gb300 import inputs
    c = dict(n=(32, 12, 20), xmin=(0.0,) * 3, h=0.05, boundary="periodic", conformal="W",
             slicing="geodesic", shift="gamma-driver", precision=precision, w_fp64_threshold=0.9)
    st = inputs.random_state(5, c["n"], c["xmin"], c["h"], amp=0.05)
    evo = B.Evolution(gpu_params(c))
    want = []
    for s in range(2):
        evo.set_state(st * (1.0 + 1e-3 * s), 0.0)
        evo.rk4_step(1)
        want.append(evo.get_state()[0])
    if staging:
        evo.enable_copy_staging()
    host_in = [_pinned(torch_cuda, evo.shape) for _ in range(2)]
    host_out = [_pinned(torch_cuda, evo.shape) for _ in range(2)]
    for s in range(2):
        host_in[s][...] = st * (1.0 + 1e-3 * s)
        B.bssn_set_state_async(evo.ctx, host_in[s], 0.0)
        evo.rk4_step(1)
        B.bssn_get_state_async(evo.ctx, host_out[s])
    B.bssn_wait_state(evo.ctx)
    for s in range(2):
        assert np.array_equal(host_out[s], want[s]), s
    # ghosts garbled on the host: the step fills them from the interior first
    bad = st.copy()
    bad[:, :3] = 7.0
    evo.set_state(bad, 0.0)
    evo.rk4_step(1)
    assert np.array_equal(evo.get_state()[0], want[0])
    evo.close()
