"""Parity of the double-word precision path (BSSN_FF: stencils and right-hand
side in double-word "float-float" arithmetic on the float32 pipe, RK4 state
and k-sum in float64) with the float64 CPU oracle, through the C ABI.

Bars, derived from the float64 bars by the ratio of unit roundoffs: a
double-word operation rounds at most a few 2^-48 of its operands (Dekker's
sum and product, Joldes-Muller-Popescu bounds), against 2^-53 for float64, a
factor 2^7 = 128 at most.
* right-hand side: the rounding-aware float64 bar, 1e-12 of the larger of the
  field's scale and the oracle's magnitude of the terms at the point
  (cases.rounding_aware_errors); the float64 kernels use 5e-4 of it, so 128x
  that still passes;
* RK4 steps: 128 x the float64 step bar of 1e-11, normwise per field.
Inputs come from the oracle or the seeded generators, never from the CUDA
path."""
import numpy as np
import pytest

import oracle as O
from cases import bl_params, gpu_params, normwise_errors, oracle_cfg, rounding_aware_errors
from paper_1111_3344_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-12
TOL_STEP = 1e-11 * 128

BL1 = dict(n=(37, 21, 19), xmin=(-4.1, -2.3, -2.2), h=0.2203, boundary="sommerfeld",
           punctures=[(1.0, 0.05, -0.02, 0.01)], r_excise=0.8, precision="ff")
CASES = {
    "bl_w_1pluslog_sommerfeld": dict(BL1, conformal="W", slicing="1+log", shift="gamma-driver", eta=2.0, q_R=1.7),
    "bl_phi_harmonic_sommerfeld": dict(BL1, conformal="phi", slicing="harmonic", shift="gamma-driver", eta=0.5),
    "random_periodic_w_geodesic": dict(n=(33, 9, 12), xmin=(-0.5, -0.2, -0.3), h=1.0 / 33, boundary="periodic",
                                       conformal="W", slicing="geodesic", precision="ff"),
    "random_periodic_phi_frozen": dict(n=(16, 40, 8), xmin=(0.0, 0.0, 0.0), h=0.05, boundary="periodic",
                                       conformal="phi", slicing="1+log", shift="frozen", precision="ff"),
    "minimal_grid": dict(n=(4, 4, 4), xmin=(-0.2, -0.2, -0.2), h=0.1, boundary="sommerfeld", conformal="W",
                         precision="ff"),
}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return torch


def _evo(case):
    from paper_1111_3344_gb300.bssn import Evolution
    return Evolution(gpu_params(case))


def _state_for(case):
    cfg = oracle_cfg(case)
    if case.get("punctures"):
        bg = O.initial_data(cfg, "bl", bl_params(case))
        return inputs.random_state(7, case["n"], case["xmin"], case["h"], amp=0.05, background=bg)
    st = inputs.random_state(11, case["n"], case["xmin"], case["h"], amp=0.1)
    return O.fill_periodic(cfg, st) if case["boundary"] == "periodic" else st


@pytest.mark.parametrize("name", list(CASES))
def test_ff_rhs_matches_oracle(torch_cuda, name):
    case = CASES[name]
    cfg = oracle_cfg(case)
    st = _state_for(case)
    want, mag = O.rhs_mag(cfg, st)
    evo = _evo(case)
    got = evo.register_to_numpy(evo.rhs(evo.numpy_to_register(st)))
    r = rounding_aware_errors(got, want, mag, TOL_RHS)
    e = normwise_errors(got, want)
    print(name, "ff rhs rounding-aware", r.max(), "normwise", e.max())
    assert r.max() <= 1.0, (dict(zip(O.FIELD_NAMES, r)), dict(zip(O.FIELD_NAMES, e)))
    evo.close()


@pytest.mark.parametrize("name", ["bl_w_1pluslog_sommerfeld", "bl_phi_harmonic_sommerfeld",
                                  "random_periodic_w_geodesic"])
def test_ff_rk4_matches_oracle(torch_cuda, name):
    case = CASES[name]
    cfg = oracle_cfg(case)
    st = _state_for(case)
    want = O.rk4(cfg, st, 3)
    evo = _evo(case)
    evo.set_state(st, 0.0)
    evo.rk4_step(3)
    got, t = evo.get_state()
    e = normwise_errors(got, want)
    print(name, "ff 3 steps normwise", e.max())
    assert e.max() <= TOL_STEP, dict(zip(O.FIELD_NAMES, e))
    assert t == pytest.approx(3 * case.get("dt", 0.25 * case["h"]))
    evo.close()


def test_ff_configurations_agree_bit_for_bit_and_are_deterministic(torch_cuda):
    """Every double-word configuration runs the same per-point arithmetic (no
    value crosses threads), so all give the same bits, run after run."""
    from paper_1111_3344_gb300 import bssn as B
    case = CASES["bl_w_1pluslog_sommerfeld"]
    st = _state_for(case)
    names = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())]
    ffc = [c for c, nm in enumerate(names) if nm.startswith("ff")]
    assert len(ffc) >= 2
    outs = []
    for c in ffc + ffc[:1]:
        evo = _evo(case)
        B.bssn_set_tile(evo.ctx, c)
        evo.set_state(st, 0.0)
        evo.rk4_step(2)
        outs.append(evo.get_state()[0])
        evo.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    # float64 and mixed configurations are refused on a double-word context
    evo = _evo(case)
    with pytest.raises(B.BssnError):
        B.bssn_set_tile(evo.ctx, names.index("32x4x1/1"))
    evo.close()


def test_ff_async_copies_match_synchronous(torch_cuda):
    """The pipelined upload / step / read-back loop with staging areas gives the
    same bits as synchronous copies (the double-word shadow of y_n is rebuilt
    after every upload)."""
    from paper_1111_3344_gb300 import bssn as B
    case = CASES["bl_w_1pluslog_sommerfeld"]
    st = _state_for(case)
    ref = _evo(case)
    outs = []
    for _ in range(2):
        ref.set_state(st, 0.0)
        ref.rk4_step(1)
        outs.append(ref.get_state()[0])
    ref.close()
    evo = _evo(case)
    evo.enable_copy_staging()
    host = [torch_cuda.empty(st.shape, dtype=torch_cuda.float64, pin_memory=True).numpy() for _ in range(2)]
    src = torch_cuda.empty(st.shape, dtype=torch_cuda.float64, pin_memory=True).numpy()
    src[...] = st
    for s in range(2):
        B.bssn_set_state_async(evo.ctx, src, 0.0)
        evo.rk4_step(1)
        B.bssn_get_state_async(evo.ctx, host[s])
    B.bssn_wait_state(evo.ctx)
    for s in range(2):
        assert np.array_equal(host[s], outs[s])
    evo.close()


def _ff_member(n, xmin, punct, boundary="sommerfeld"):
    return dict(n=n, xmin=xmin, h=0.2, boundary=boundary, conformal="W", slicing="1+log",
                shift="gamma-driver", eta=2.0, punctures=punct, precision="ff")


def test_ff_batch_matches_single_grid_bit_for_bit(torch_cuda):
    """A double-word batch runs the single-grid double-word point functions, so
    each member's state after its steps is the same, bit for bit, alone in a
    batch, in the mix with others, and through a bssn_ctx: the full-tile member
    (n0 a multiple of 32, n1 of 4) against the full-row configuration of the
    same register cap, the ragged one against the every-stencil configuration.
    The full-tile member is also checked against the oracle (three steps)."""
    from paper_1111_3344_gb300 import bssn as B
    full = _ff_member((32, 16, 20), (-3.2, -1.6, -2.0), [(0.8, 0.1, 0.0, 0.0)])
    ragged = _ff_member((33, 17, 21), (-3.3, -1.7, -2.1), [(0.6, 0.2, 0.1, 0.0)])
    per = _ff_member((16, 12, 20), (0.0, 0.0, 0.0), [], boundary="periodic")
    cases = [full, ragged, per]
    states = []
    for c in cases:
        if c["punctures"]:
            cfg = oracle_cfg(c)
            bg = O.initial_data(cfg, "bl", bl_params(c))
            states.append(inputs.random_state(17, c["n"], c["xmin"], c["h"], amp=0.03, background=bg))
        else:
            states.append(O.fill_periodic(oracle_cfg(c), inputs.random_state(5, c["n"], c["xmin"], c["h"],
                                                                            amp=0.05)))
    params = [gpu_params(c) for c in cases]
    lib = B.load()
    bnames = [lib.bssn_batch_tile_name(i).decode() for i in range(lib.bssn_batch_tile_count())]

    def run(idx):
        b = B.Batch("ff", pool_bytes=sum(B.Batch.member_bytes(params[i]) for i in idx) + (16 << 20),
                    max_members=4)
        b.set_tile(bnames.index("fftiles32x4x1/8+8"))
        ids = [b.add(params[i]) for i in idx]
        for m, i in zip(ids, idx):
            b.set_state(m, states[i], 0.0)
        b.step(3)
        out = {i: b.get_state(m)[0] for m, i in zip(ids, idx)}
        b.close()
        return out

    mix = run([0, 1, 2])
    for i in range(3):
        assert np.array_equal(run([i])[i], mix[i]), i
    names = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())]
    for i, tile in ((0, "ffrows32x4x1/8"), (1, "ff32x4x1/1")):
        evo = _evo(cases[i])
        B.bssn_set_tile(evo.ctx, names.index(tile))
        evo.set_state(states[i], 0.0)
        evo.rk4_step(3)
        assert np.array_equal(evo.get_state()[0], mix[i]), i
        evo.close()
    e = normwise_errors(mix[0], O.rk4(oracle_cfg(full), states[0], 3))
    assert e.max() <= TOL_STEP, dict(zip(O.FIELD_NAMES, e))
    # float64 and mixed configurations are refused on a double-word batch
    b = B.Batch("ff", pool_bytes=B.Batch.member_bytes(params[0]) + (16 << 20), max_members=2)
    with pytest.raises(B.BssnError):
        b.set_tile(bnames.index("tma32x4x1/2"))
    b.close()


def test_ff_server_same_alone_and_in_the_mix(torch_cuda):
    """The continuous-batching server in double-word precision: requests give the
    same constraint norms, bit for bit, alone and admitted while others run."""
    import time
    from paper_1111_3344_gb300.bssn import Params, Server

    def req(n):
        L = 4.0
        h = 2 * L / n
        return Params(n=(n, n, n), xmin=(-L,) * 3, h=h, boundary="sommerfeld", conformal="W",
                      dt=0.25 * h, precision="ff", r_excise=0.5)

    reqs = [(24, [1, 0.5, 0.3, 0.0, 0.0], 6), (32, [2, 0.6, 1.0, 0.0, 0.0, 0.4, -1.5, 0.0, 0.0], 4),
            (20, [1, 1.0, 0.0, 0.0, 0.0], 8)]
    alone = {}
    for i, (n, p, steps) in enumerate(reqs):
        s = Server("ff", budget_bytes=1 << 28)
        st, norms, _ = s.wait(s.submit(req(n), "bl", p, steps))
        assert st == 0
        alone[i] = norms
        s.close()
    s = Server("ff", budget_bytes=1 << 29)
    long_t = s.submit(req(24), "bl", reqs[0][1], 200)
    t0 = time.time()
    while s.stats()["resident"] < 1 and time.time() - t0 < 30:
        time.sleep(0.001)
    tickets = [s.submit(req(n), "bl", p, steps) for (n, p, steps) in reqs]
    for i, t in enumerate(tickets):
        st, norms, _ = s.wait(t)
        assert st == 0 and np.array_equal(norms, alone[i]), i
    assert s.wait(long_t)[0] == 0
    s.close()
