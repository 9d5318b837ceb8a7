"""Batched evolutions (one persistent launch per RK4 stage, CUDA graph) and the
continuous-batching server.

The bar: a member's state after n steps is bit-identical whether it runs alone
in a batch or together with other members (the same kernel runs the same
per-point arithmetic; the work-list only decides which block does which tile),
and it matches the single-evolution path to the parity tolerance of the
precision (float64: 1e-11 normwise; mixed: 1e-6)."""
import time

import numpy as np
import pytest

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


def _members(precision):
    bl1 = dict(n=(24, 20, 28), xmin=(-3.0, -2.5, -3.5), h=0.25, boundary="sommerfeld", conformal="W",
               slicing="1+log", shift="gamma-driver", eta=2.0, punctures=[(1.0, 0.05, 0.0, 0.0)],
               precision=precision, w_fp64_threshold=0.3)
    bl2 = dict(n=(33, 17, 21), xmin=(-4.0, -2.1, -2.6), h=0.25, boundary="sommerfeld", conformal="W",
               slicing="1+log", shift="gamma-driver", eta=1.0,
               punctures=[(0.6, 1.0, 0.0, 0.0), (0.4, -1.5, 0.0, 0.0)], precision=precision,
               w_fp64_threshold=0.3)
    gw = dict(n=(24, 24, 24), xmin=(-0.5,) * 3, h=1 / 24, boundary="periodic", conformal="phi",
              slicing="harmonic", shift="frozen", precision=precision)
    rnd = dict(n=(16, 12, 20), xmin=(0.0,) * 3, h=0.05, boundary="periodic", conformal="W",
               slicing="geodesic", shift="gamma-driver", precision=precision, w_fp64_threshold=0.9)
    return [bl1, bl2, gw, rnd]


def _initial(case):
    if case.get("punctures"):
        return ("bl", bl_params(case))
    if case["slicing"] == "harmonic":
        return ("gauge_wave", [0.01, 1.0])
    return ("state", inputs.random_state(5, case["n"], case["xmin"], case["h"], amp=0.05))


def _load(batch, mid, case):
    kind, p = _initial(case)
    if kind == "state":
        batch.set_state(mid, p, 0.0)
    else:
        batch.set_initial_data(mid, kind, p)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alone_equals_in_the_mix(torch_cuda, precision):
    from paper_1111_3344_gb300.bssn import Batch, Evolution
    cases = _members(precision)
    steps = 3
    mix = Batch(precision, pool_bytes=1 << 30)
    ids = [mix.add(gpu_params(c)) for c in cases]
    for mid, c in zip(ids, cases):
        _load(mix, mid, c)
    mix.step(steps)
    got_mix = [mix.get_state(m)[0] for m in ids]
    norms_mix = [mix.constraints(m) for m in ids]
    tile = 0
    for c, gm, nm in zip(cases, got_mix, norms_mix):
        alone = Batch(precision, pool_bytes=1 << 29)
        mid = alone.add(gpu_params(c))
        _load(alone, mid, c)
        alone.step(steps)
        ga, t = alone.get_state(mid)
        assert np.array_equal(ga, gm)
        assert np.array_equal(alone.constraints(mid), nm)
        assert t == pytest.approx(steps * gpu_params(c).dt)
        alone.close()
        # and against the single-evolution path
        evo = Evolution(gpu_params(c))
        kind, p = _initial(c)
        if kind == "state":
            evo.set_state(p, 0.0)
        else:
            evo.set_initial_data(kind, p)
        evo.rk4_step(steps)
        e = normwise_errors(gm, evo.get_state()[0])
        assert e.max() <= (1e-11 if precision == "fp64" else 1e-4), e.max()
        evo.close()
    mix.close()


def test_batch_matches_oracle_fp64(torch_cuda):
    from paper_1111_3344_gb300.bssn import Batch
    c = _members("fp64")[1]
    b = Batch("fp64", pool_bytes=1 << 28)
    mid = b.add(gpu_params(c))
    b.set_initial_data(mid, "bl", bl_params(c))
    b.step(2)
    got, _ = b.get_state(mid)
    cfg = oracle_cfg(c)
    want = O.rk4(cfg, O.initial_data(cfg, "bl", bl_params(c)), 2)
    assert normwise_errors(got, want).max() <= 1e-11


def test_membership_changes_between_steps(torch_cuda):
    """Members join and leave between steps without re-capture; a member that
    stays is unaffected by the others coming and going."""
    from paper_1111_3344_gb300.bssn import Batch
    cs = _members("mixed")
    b = Batch("mixed", pool_bytes=1 << 30)
    a = b.add(gpu_params(cs[0]))
    _load(b, a, cs[0])
    b.step(2)
    x = b.add(gpu_params(cs[1]))
    _load(b, x, cs[1])
    b.step(2)
    b.remove(x)
    y = b.add(gpu_params(cs[2]))
    _load(b, y, cs[2])
    b.step(2)
    got, t = b.get_state(a)
    ref = Batch("mixed", pool_bytes=1 << 29)
    r = ref.add(gpu_params(cs[0]))
    _load(ref, r, cs[0])
    ref.step(6)
    assert np.array_equal(got, ref.get_state(r)[0])


def test_pool_exhaustion_and_precision_mismatch(torch_cuda):
    from paper_1111_3344_gb300.bssn import Batch, BssnError
    c = _members("fp64")[0]
    need = Batch.member_bytes(gpu_params(c))
    b = Batch("fp64", pool_bytes=need + (2 << 20), max_members=4)
    b.add(gpu_params(c))
    with pytest.raises(BssnError) as e:
        b.add(gpu_params(c))
    assert e.value.status == 2
    with pytest.raises(BssnError) as e:
        b.add(gpu_params(dict(c, precision="mixed")))
    assert e.value.status == 1


def test_batch_autotune_keeps_results(torch_cuda):
    from paper_1111_3344_gb300.bssn import Batch
    cs = _members("mixed")
    outs = []
    for tune in (False, True):
        b = Batch("mixed", pool_bytes=1 << 30)
        ids = [b.add(gpu_params(c)) for c in cs]
        for m, c in zip(ids, cs):
            _load(b, m, c)
        if tune:
            best, times = b.autotune(reps=1)
            assert len(times) >= 2
        b.step(2)
        outs.append([b.get_state(m)[0] for m in ids])
    for x, y in zip(*outs):
        assert normwise_errors(x, y).max() <= 1e-4


# ------------------------------------------------------------------ server

def _req(n, L=6.0, precision="mixed"):
    from paper_1111_3344_gb300.bssn import Params
    h = 2 * L / n
    return Params(n=(n,) * 3, xmin=(-L,) * 3, h=h, boundary="sommerfeld", conformal="W",
                  slicing="1+log", shift="gamma-driver", eta=2.0, dt=0.25 * h, precision=precision,
                  w_fp64_threshold=0.2, r_excise=1.0)


@pytest.mark.parametrize("policy", ["all", "shortest"])
def test_server_results_same_alone_and_in_the_mix(torch_cuda, policy):
    """Each request's constraint norms are the same bits alone and arriving
    while another request runs, whether every resident request steps every
    time or the shortest remaining work goes first (min_points small enough
    that requests are held while others step)."""
    from paper_1111_3344_gb300.bssn import Server
    reqs = [(24, [1, 0.5, 0.3, 0.0, 0.0], 12), (32, [2, 0.6, 1.0, 0.0, 0.0, 0.4, -1.5, 0.0, 0.0], 5),
            (20, [1, 1.0, 0.0, 0.0, 0.0], 20), (28, [1, 0.7, 0.0, 0.2, 0.0], 8)]
    alone = {}
    for i, (n, p, steps) in enumerate(reqs):
        s = Server("mixed", budget_bytes=1 << 28)
        t = s.submit(_req(n), "bl", p, steps)
        st, norms, lat = s.wait(t)
        assert st == 0 and lat > 0
        alone[i] = norms
        s.close()
    s = Server("mixed", budget_bytes=1 << 29)
    s.set_policy(policy, min_points=20 ** 3)
    long_t = s.submit(_req(24), "bl", reqs[0][1], 400)   # keeps the batch busy
    t0 = time.time()
    while s.stats()["resident"] < 1 and time.time() - t0 < 30:
        time.sleep(0.001)
    tickets = [s.submit(_req(n), "bl", p, steps) for (n, p, steps) in reqs]  # arrive while it runs
    res = [s.wait(t) for t in tickets]
    assert s.poll(long_t) is None or s.poll(long_t)[0] == 0
    for i, (st, norms, lat) in enumerate(res):
        assert st == 0
        assert np.array_equal(norms, alone[i]), i
    st, _, _ = s.wait(long_t)
    assert st == 0
    stats = s.stats()
    assert stats["completed"] == 5 and stats["failed"] == 0 and stats["point_updates"] > 0
    # every request advanced exactly its own steps
    assert stats["point_updates"] == 24 ** 3 * 400 + sum(n ** 3 * steps for n, _, steps in reqs)
    s.close()


def test_batch_hold_leaves_member_unchanged(torch_cuda):
    """A held member keeps its state and time while the others step; resumed,
    it reaches the same bits as a member that was never held."""
    from paper_1111_3344_gb300.bssn import Batch
    cs = _members("mixed")[:2]
    b = Batch("mixed", pool_bytes=1 << 29)
    ids = [b.add(gpu_params(c)) for c in cs]
    for m, c in zip(ids, cs):
        _load(b, m, c)
    before, t0 = b.get_state(ids[0])
    b.hold(ids[0])
    b.step(3)
    held, t1 = b.get_state(ids[0])
    assert np.array_equal(before, held) and t1 == t0
    b.hold(ids[0], False)
    b.step(2)
    got = b.get_state(ids[0])[0]
    b.close()
    ref = Batch("mixed", pool_bytes=1 << 29)
    rid = ref.add(gpu_params(cs[0]))
    _load(ref, rid, cs[0])
    ref.step(2)
    assert np.array_equal(ref.get_state(rid)[0], got)
    ref.close()


def test_server_budget_and_failure_isolation(torch_cuda):
    from paper_1111_3344_gb300.bssn import BssnError, Server
    s = Server("mixed", budget_bytes=1 << 27)
    with pytest.raises(BssnError) as e:   # larger than the whole budget
        s.submit(_req(160), "bl", [1, 1.0, 0.0, 0.0, 0.0], 10)
    assert e.value.status == 1
    good = s.submit(_req(20), "bl", [1, 1.0, 0.0, 0.0, 0.0], 6)
    bad = s.submit(_req(20), "bl", [1, float("nan"), 0.0, 0.0, 0.0], 6)
    good2 = s.submit(_req(24), "bl", [1, 0.8, 0.1, 0.0, 0.0], 6)
    assert s.wait(good)[0] == 0
    assert s.wait(bad)[0] == 7          # BSSN_EFAILED, only for that request
    assert s.wait(good2)[0] == 0
    st = s.stats()
    assert st["failed"] == 1 and st["completed"] == 3
    s.close()


def test_batch_full_rows_fp64(torch_cuda):
    """A float64 member whose tiles are all full (x extent a multiple of 32,
    y and z of every tile shape) takes the full-block point function (first
    differences shared across the warp's lanes and across rows through shared
    memory); next to a member with ragged tiles it still matches the oracle and
    itself alone, bit for bit."""
    from paper_1111_3344_gb300.bssn import Batch
    rows = dict(n=(64, 16, 12), xmin=(-8.0, -2.0, -1.5), h=0.25, boundary="sommerfeld", conformal="W",
                slicing="1+log", shift="gamma-driver", eta=2.0, punctures=[(1.0, 0.05, 0.0, 0.0)],
                precision="fp64", w_fp64_threshold=0.3)
    ragged = _members("fp64")[1]
    mix = Batch("fp64", pool_bytes=1 << 29)
    ids = [mix.add(gpu_params(c)) for c in (rows, ragged)]
    for mid, c in zip(ids, (rows, ragged)):
        mix.set_initial_data(mid, "bl", bl_params(c))
    mix.step(2)
    got = mix.get_state(ids[0])[0]
    alone = Batch("fp64", pool_bytes=1 << 28)
    aid = alone.add(gpu_params(rows))
    alone.set_initial_data(aid, "bl", bl_params(rows))
    alone.step(2)
    assert np.array_equal(alone.get_state(aid)[0], got)
    alone.close()
    cfg = oracle_cfg(rows)
    want = O.rk4(cfg, O.initial_data(cfg, "bl", bl_params(rows)), 2)
    assert normwise_errors(got, want).max() <= 1e-11
    cfg = oracle_cfg(ragged)
    want = O.rk4(cfg, O.initial_data(cfg, "bl", bl_params(ragged)), 2)
    assert normwise_errors(mix.get_state(ids[1])[0], want).max() <= 1e-11
    mix.close()


def test_batch_fp64_configurations_agree_bitwise(torch_cuda):
    """Every float64 tile configuration of a batch -- the persistent kernels,
    whose per-tile body is a call of its own, and the one-block-per-tile
    kernels -- runs the same point functions on a member with full tiles and
    on members with ragged ones: two steps give the same bits whichever
    configuration runs them."""
    from paper_1111_3344_gb300 import bssn as B
    from paper_1111_3344_gb300.bssn import Batch
    rows = dict(n=(64, 16, 8), xmin=(-8.0, -2.0, -1.0), h=0.25, boundary="sommerfeld", conformal="W",
                slicing="1+log", shift="gamma-driver", eta=2.0, punctures=[(1.0, 0.05, 0.0, 0.0)],
                precision="fp64", w_fp64_threshold=0.3)
    cases = [rows] + _members("fp64")[:3]
    lib = B.load()
    names = [lib.bssn_batch_tile_name(c).decode() for c in range(lib.bssn_batch_tile_count())]
    # (the per-member configuration runs the single-grid kernels: its own test)
    fp64_cfgs = [c for c, nm in enumerate(names) if not nm.startswith(("tma", "ff", "members"))]
    assert "32x4x1/3" in names and "tiles32x4x1/2" in names
    ref = None
    for c in fp64_cfgs:
        b = Batch("fp64", pool_bytes=1 << 29)
        ids = [b.add(gpu_params(cs)) for cs in cases]
        for m, cs in zip(ids, cases):
            _load(b, m, cs)
        b.set_tile(c)
        b.step(2)
        got = [b.get_state(m)[0] for m in ids]
        b.close()
        if ref is None:
            ref = got
            continue
        for x, y in zip(ref, got):
            assert np.array_equal(x, y), names[c]


@pytest.mark.parametrize("tile", ["tma32x4x1/2", "tma11_32x8x1/1"])
def test_batch_tma_tile_matches_single_grid_tma(torch_cuda, tile):
    """The TMA-staged batched kernels (mixed; 8 staged fields on 32x4x1 tiles,
    or 11 on 32x8x1 tiles): each member's state is the same bit for bit alone
    and in the mix, and matches the single-grid evolution on the same
    TMA-staged tile to the mixed parity bar (the same per-point source,
    compiled into two kernels whose floating-point contractions may differ);
    the float64 batch refuses the tile."""
    from paper_1111_3344_gb300 import bssn as B
    n_cfg = B.load().bssn_batch_tile_count()
    names = [B.load().bssn_batch_tile_name(c).decode() for c in range(n_cfg)]
    tma = names.index(tile)
    cases = _members("mixed")
    steps = 3
    mix = B.Batch("mixed", pool_bytes=1 << 30)
    ids = [mix.add(gpu_params(c)) for c in cases]
    for mid, c in zip(ids, cases):
        _load(mix, mid, c)
    mix.set_tile(tma)
    mix.step(steps)
    single_tma = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())].index(tile)
    for mid, c in zip(ids, cases):
        got, _ = mix.get_state(mid)
        evo = B.Evolution(gpu_params(c))
        kind, p = _initial(c)
        if kind == "state":
            evo.set_state(p, 0.0)
        else:
            evo.set_initial_data(kind, p)
        B.bssn_set_tile(evo.ctx, single_tma)
        evo.rk4_step(steps)
        e = normwise_errors(got, evo.get_state()[0])
        assert e.max() <= 1e-4, (c["n"], e.max())
        evo.close()
        alone = B.Batch("mixed", pool_bytes=1 << 29)
        aid = alone.add(gpu_params(c))
        _load(alone, aid, c)
        alone.set_tile(tma)
        alone.step(steps)
        assert np.array_equal(alone.get_state(aid)[0], got)
        alone.close()
    mix.close()
    f64 = B.Batch("fp64", pool_bytes=1 << 28)
    with pytest.raises(Exception):
        f64.set_tile(tma)
    f64.close()


SINGLE_TILE = {"fp64": "32x4x1/1", "mixed": "tma11_32x8x1/1", "ff": "ffrows32x4x1/8"}


@pytest.mark.parametrize("precision,tile", [("fp64", "members"), ("mixed", "members"), ("ff", "members"),
                                            ("ff", "members1"), ("mixed", "members4")])
def test_members_configuration_equals_single_grid(torch_cuda, precision, tile):
    """The per-member batch configuration launches each member's stages and
    boundaries with the single-grid kernels, the members' chains side by side
    on auxiliary streams: every member's state after two steps is the same
    bits as a single-grid evolution on the same tile, and the same alone as
    in the mix (members with full and with ragged tiles, a periodic one)."""
    from paper_1111_3344_gb300 import bssn as B
    from paper_1111_3344_gb300.bssn import Batch
    rows = dict(n=(64, 16, 8), xmin=(-8.0, -2.0, -1.0), h=0.25, boundary="sommerfeld", conformal="W",
                slicing="1+log", shift="gamma-driver", eta=2.0, punctures=[(1.0, 0.05, 0.0, 0.0)],
                precision=precision, w_fp64_threshold=0.3)
    cases = [rows] + _members(precision)[:3]
    lib = B.load()
    bnames = [lib.bssn_batch_tile_name(c).decode() for c in range(lib.bssn_batch_tile_count())]
    snames = [B.bssn_tile_name(c) for c in range(B.bssn_tile_count())]
    b = Batch(precision, pool_bytes=1 << 30)
    ids = [b.add(gpu_params(cs)) for cs in cases]
    for m, cs in zip(ids, cases):
        _load(b, m, cs)
    b.set_tile(bnames.index(tile))
    b.step(2)
    got = [b.get_state(m)[0] for m in ids]
    b.close()
    for cs, g in zip(cases, got):
        evo = B.Evolution(gpu_params(cs))
        kind, p = _initial(cs)
        if kind == "state":
            evo.set_state(p, 0.0)
        else:
            evo.set_initial_data(kind, p)
        B.bssn_set_tile(evo.ctx, snames.index(SINGLE_TILE[precision]))
        evo.rk4_step(2)
        assert np.array_equal(evo.get_state()[0], g), cs["n"]
        evo.close()
    alone = Batch(precision, pool_bytes=1 << 29)
    aid = alone.add(gpu_params(cases[1]))
    _load(alone, aid, cases[1])
    alone.set_tile(bnames.index(tile))
    alone.step(2)
    assert np.array_equal(alone.get_state(aid)[0], got[1])
    alone.close()
