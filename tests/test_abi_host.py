"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/bssn.h declares, and validates parameters."""
import math
import os
import re

import pytest

from paper_1111_3344_gb300 import bssn as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bssn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bssn_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = B.load()
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.exported_symbols())


def test_layout_and_required_bytes():
    p = B.Params(n=(128, 128, 128), xmin=(-8.0,) * 3, h=0.125, boundary="sommerfeld")
    lay = B.bssn_layout_of(p)
    assert lay["stored"] == (134, 134, 134)
    assert lay["pitch"] % 8 == 0 and lay["pitch"] >= 134
    assert lay["field_stride"] == lay["plane"] * 134 and lay["plane"] == lay["pitch"] * 134
    nb = B.bssn_required_bytes(p)
    # y_n, acc, two stage buffers and the boundary-anchor buffer
    assert nb >= 5 * 24 * lay["field_stride"] * 8
    p2 = B.Params(n=(128, 128, 128), xmin=(-8.0,) * 3, h=0.125, boundary="periodic")
    assert B.bssn_required_bytes(p2) < nb


@pytest.mark.parametrize("bad", [
    dict(n=(3, 8, 8)), dict(n=(8, 8, 4097)), dict(h=0.0), dict(h=math.nan),
    dict(boundary="periodic", dt=math.inf), dict(w_floor=0.0),
])
def test_invalid_params_rejected(bad):
    kw = dict(n=(8, 8, 8), xmin=(0.0,) * 3, h=0.1)
    kw.update(bad)
    p = B.Params(**kw)
    with pytest.raises(B.BssnError) as e:
        B.bssn_layout_of(p)
    assert e.value.status == 1
    with pytest.raises(B.BssnError):
        B.bssn_required_bytes(p)


def test_alloc_rejects_null_and_small_memory():
    p = B.Params(n=(8, 8, 8), xmin=(0.0,) * 3, h=0.1)
    with pytest.raises(B.BssnError) as e:
        B.bssn_alloc(p, 0, 1 << 30, 0)
    assert e.value.status == 1
    with pytest.raises(B.BssnError) as e:
        B.bssn_alloc(p, 256, 16, 0)  # never dereferenced: size check fails first
    assert e.value.status == 2


def test_staging_bytes():
    """bssn_staging_bytes: two areas (upload, read-back), each the state in the
    unpadded host layout rounded up to 256 bytes; 0 on bad parameters."""
    import ctypes
    lib = B.load()
    p = B.Params(n=(37, 21, 19), xmin=(0.0,) * 3, h=0.1, boundary="sommerfeld")
    c = p.c()
    n = int(lib.bssn_staging_bytes(ctypes.byref(c)))
    area = 24 * (37 + 6) * (21 + 6) * (19 + 6) * 8
    assert n == 2 * ((area + 255) // 256 * 256)
    bad = B.Params(n=(3, 8, 8), xmin=(0.0,) * 3, h=0.1).c()
    assert int(lib.bssn_staging_bytes(ctypes.byref(bad))) == 0


def test_batch_table_bytes_grow_with_members():
    """The batch tables (member table with one tensor map per stage, work list,
    error word) grow linearly with max_members; 0 outside 1..256
    (BSSN_BATCH_MAX_MEMBERS)."""
    lib = B.load()
    t1, t2, t64 = (int(lib.bssn_batch_table_bytes(m)) for m in (1, 2, 64))
    assert 0 < t1 < t2 < t64
    assert (t64 - t2) >= 62 * 4 * 128  # at least the four 128-byte tensor maps per member
    assert int(lib.bssn_batch_table_bytes(256)) > t64
    assert int(lib.bssn_batch_table_bytes(0)) == 0 and int(lib.bssn_batch_table_bytes(257)) == 0


def _select_reference(work, pts, min_points):
    """The shortest-work-first rule written out: order by remaining work (ties
    by index), take requests until their points reach min_points, at least
    one."""
    order = sorted(range(len(work)), key=lambda i: (work[i], i))
    sel, acc = [0] * len(work), 0.0
    for k, i in enumerate(order):
        if k > 0 and acc >= min_points:
            break
        sel[i] = 1
        acc += pts[i]
    return sel


def test_serve_select_shortest_work_first():
    """bssn_serve_select, the server's shortest-work-first choice, on host
    arrays: the shortest request alone when min_points is 0; the shortest
    ones until they hold min_points; everything when min_points exceeds the
    total; ties by index; and the rule restated above on seeded random sets."""
    import numpy as np
    assert list(B.bssn_serve_select([], [], 1.0)) == []
    work = [50.0, 10.0, 30.0, 20.0]
    pts = [5.0, 1.0, 3.0, 2.0]
    assert list(B.bssn_serve_select(work, pts, 0.0)) == [0, 1, 0, 0]
    assert list(B.bssn_serve_select(work, pts, 2.5)) == [0, 1, 0, 1]  # 1 + 2 >= 2.5
    assert list(B.bssn_serve_select(work, pts, 3.0)) == [0, 1, 0, 1]
    assert list(B.bssn_serve_select(work, pts, 3.5)) == [0, 1, 1, 1]
    assert list(B.bssn_serve_select(work, pts, 1e9)) == [1, 1, 1, 1]
    assert list(B.bssn_serve_select([7.0, 7.0, 7.0], [1.0, 1.0, 1.0], 1.5)) == [1, 1, 0]
    rng = np.random.default_rng(3344)
    for _ in range(200):
        n = int(rng.integers(1, 40))
        w = list(rng.integers(1, 20, n).astype(float))  # repeated values exercise the ties
        p = list(rng.integers(1, 9, n).astype(float))
        m = float(rng.uniform(0, sum(p) * 1.2))
        assert list(B.bssn_serve_select(w, p, m)) == _select_reference(w, p, m)


@pytest.mark.parametrize("n", [(4096, 4096, 4096), (4096, 4, 4), (4, 4096, 4096)])
def test_sizes_at_the_largest_grids(n):
    """At the largest accepted sides (4096) the layout and the byte counts are
    formed in 64-bit arithmetic: a float64 register of 24 fields exceeds 2^32
    points and 2^40 bytes at 4096^3 and must not wrap."""
    p = B.Params(n=n, xmin=(0.0,) * 3, h=0.1, boundary="sommerfeld")
    lay = B.bssn_layout_of(p)
    assert lay["stored"] == tuple(x + 6 for x in n)
    assert lay["pitch"] >= n[0] + 6 and lay["plane"] == lay["pitch"] * (n[1] + 6)
    assert lay["field_stride"] == lay["plane"] * (n[2] + 6)
    nb = B.bssn_required_bytes(p)
    assert nb >= 5 * 24 * lay["field_stride"] * 8
    if n == (4096, 4096, 4096):
        assert nb > 1 << 42
