"""ctypes binding of libbssn (include/bssn.h): the same entry points with the
same names, argument marshalling only.  Every step of the evolution runs in
the CUDA library; PyTorch supplies device memory and the stream.

There is no fallback: if the library is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

NUM_FIELDS = 24
GHOST = 3

BC = {"periodic": 0, "sommerfeld": 1}
CONFORMAL = {"phi": 0, "W": 1}
SLICING = {"1+log": 0, "harmonic": 1, "geodesic": 2}
SHIFT = {"gamma-driver": 0, "frozen": 1}
PRECISION = {"fp64": 0, "mixed": 1, "ff": 2}
ID_KIND = {"flat": 0, "gauge_wave": 1, "bl": 2, "kasner": 3}
SERVE_POLICY = {"all": 0, "shortest": 1}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EAGAIN", 5: "ETIMEOUT",
          6: "ENOTFOUND", 7: "EFAILED"}


class BssnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class bssn_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("ghost", ctypes.c_int32),
        ("xmin", ctypes.c_double * 3),
        ("h", ctypes.c_double),
        ("boundary", ctypes.c_int32),
        ("conformal", ctypes.c_int32),
        ("slicing", ctypes.c_int32),
        ("shift", ctypes.c_int32),
        ("eta", ctypes.c_double),
        ("q_R", ctypes.c_double),
        ("ko_eps", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("ksum_fp64", ctypes.c_int32),
        ("w_fp64_threshold", ctypes.c_double),
        ("r_excise", ctypes.c_double),
        ("w_floor", ctypes.c_double),
    ]


class bssn_layout(ctypes.Structure):
    _fields_ = [
        ("stored", ctypes.c_int32 * 3),
        ("ghost", ctypes.c_int32),
        ("pitch", ctypes.c_int64),
        ("plane", ctypes.c_int64),
        ("field_stride", ctypes.c_int64),
        ("register_elems", ctypes.c_int64),
    ]


@dataclass
class Params:
    """Python mirror of bssn_params with readable enum values."""
    n: tuple = (24, 24, 24)
    xmin: tuple = (-0.5, -0.5, -0.5)
    h: float = 1.0 / 24.0
    boundary: str = "periodic"
    conformal: str = "W"
    slicing: str = "1+log"
    shift: str = "gamma-driver"
    eta: float = 2.0
    q_R: float = math.inf
    ko_eps: float = 0.1
    dt: float = 0.25 / 24.0
    precision: str = "fp64"
    ksum_fp64: bool = False
    w_fp64_threshold: float = 0.0
    r_excise: float = 1.0
    w_floor: float = 1e-10

    def c(self) -> bssn_params:
        p = bssn_params()
        for d in range(3):
            p.n[d] = int(self.n[d])
            p.xmin[d] = float(self.xmin[d])
        p.ghost = GHOST
        p.h = float(self.h)
        p.boundary = BC[self.boundary]
        p.conformal = CONFORMAL[self.conformal]
        p.slicing = SLICING[self.slicing]
        p.shift = SHIFT[self.shift]
        p.eta = float(self.eta)
        p.q_R = float(self.q_R)
        p.ko_eps = float(self.ko_eps)
        p.dt = float(self.dt)
        p.precision = PRECISION[self.precision]
        p.ksum_fp64 = 1 if self.ksum_fp64 else 0
        p.w_fp64_threshold = float(self.w_fp64_threshold)
        p.r_excise = float(self.r_excise)
        p.w_floor = float(self.w_floor)
        return p


_lib = None

# (name, argtypes, restype) of every exported entry point
_SIGS = [
    ("bssn_last_error", [], ctypes.c_char_p),
    ("bssn_layout_of", [ctypes.POINTER(bssn_params), ctypes.POINTER(bssn_layout)], ctypes.c_int),
    ("bssn_required_bytes", [ctypes.POINTER(bssn_params)], ctypes.c_size_t),
    ("bssn_alloc", [ctypes.POINTER(bssn_params), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                    ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    ("bssn_free", [ctypes.c_void_p], ctypes.c_int),
    ("bssn_state_ptr", [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    ("bssn_set_initial_data", [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                               ctypes.c_int32], ctypes.c_int),
    ("bssn_rhs", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    ("bssn_rk4_step", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_constraints", [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_get_state", [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_set_state", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double], ctypes.c_int),
    ("bssn_get_state_async", [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_set_state_async", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double], ctypes.c_int),
    ("bssn_wait_state", [ctypes.c_void_p], ctypes.c_int),
    ("bssn_staging_bytes", [ctypes.c_void_p], ctypes.c_size_t),
    ("bssn_set_staging", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    ("bssn_profile", [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_set_adm", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double], ctypes.c_int),
    ("bssn_set_punctures", [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32], ctypes.c_int),
    ("bssn_track_punctures", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_get_punctures", [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)],
     ctypes.c_int),
    ("bssn_adm_integrals", [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_psi4", [ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    ("bssn_set_matter", [ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    ("bssn_tile_count", [], ctypes.c_int32),
    ("bssn_tile_name", [ctypes.c_int32], ctypes.c_char_p),
    ("bssn_set_tile", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_autotune", [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                       ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_constraints_noalloc", [ctypes.POINTER(bssn_params), ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_test_stall_tma", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_peak_probe", [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                         ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
]


_SIGS += [
    ("bssn_batch_table_bytes", [ctypes.c_int32], ctypes.c_size_t),
    ("bssn_batch_member_bytes", [ctypes.POINTER(bssn_params)], ctypes.c_size_t),
    ("bssn_batch_create", [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    ("bssn_batch_free", [ctypes.c_void_p], ctypes.c_int),
    ("bssn_batch_add", [ctypes.c_void_p, ctypes.POINTER(bssn_params), ctypes.POINTER(ctypes.c_int32)],
     ctypes.c_int),
    ("bssn_batch_remove", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_batch_set_initial_data", [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int32], ctypes.c_int),
    ("bssn_batch_set_state", [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double],
     ctypes.c_int),
    ("bssn_batch_get_state", [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_batch_step", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_batch_constraints", [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)],
     ctypes.c_int),
    ("bssn_batch_hold", [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
    ("bssn_batch_test_stall_tma", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_batch_tile_count", [], ctypes.c_int32),
    ("bssn_batch_tile_name", [ctypes.c_int32], ctypes.c_char_p),
    ("bssn_batch_set_tile", [ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    ("bssn_batch_autotune", [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_server_create", [ctypes.c_int32, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                            ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    ("bssn_submit", [ctypes.c_void_p, ctypes.POINTER(bssn_params), ctypes.c_int32,
                     ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int32,
                     ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    ("bssn_poll", [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                   ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_poll_detail", [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_server_stats", [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("bssn_server_set_policy", [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double], ctypes.c_int),
    ("bssn_serve_select", [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.c_double, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int32),
    ("bssn_server_destroy", [ctypes.c_void_p], ctypes.c_int),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbssn.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libbssn.so not found at {_build.LIB}; run paper_1111_3344_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, args, res in _SIGS:
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return [s[0] for s in _SIGS]


def _check(status):
    if status != 0:
        raise BssnError(status, load().bssn_last_error().decode())


def _dbl_array(vals):
    arr = (ctypes.c_double * max(1, len(vals)))(*[float(v) for v in vals])
    return arr


# ---------------------------------------------------------------- raw ABI
def bssn_layout_of(params: Params) -> dict:
    p = params.c()
    lay = bssn_layout()
    _check(load().bssn_layout_of(ctypes.byref(p), ctypes.byref(lay)))
    return {"stored": tuple(lay.stored), "ghost": lay.ghost, "pitch": lay.pitch,
            "plane": lay.plane, "field_stride": lay.field_stride,
            "register_elems": lay.register_elems}


def bssn_required_bytes(params: Params) -> int:
    p = params.c()
    n = load().bssn_required_bytes(ctypes.byref(p))
    if n == 0:
        raise BssnError(1, load().bssn_last_error().decode())
    return int(n)


def bssn_alloc(params: Params, d_mem: int, nbytes: int, stream: int) -> int:
    p = params.c()
    out = ctypes.c_void_p()
    _check(load().bssn_alloc(ctypes.byref(p), ctypes.c_void_p(d_mem), nbytes,
                             ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def bssn_free(ctx: int):
    _check(load().bssn_free(ctypes.c_void_p(ctx)))


def bssn_state_ptr(ctx: int) -> int:
    out = ctypes.c_void_p()
    _check(load().bssn_state_ptr(ctypes.c_void_p(ctx), ctypes.byref(out)))
    return out.value


def bssn_set_initial_data(ctx: int, kind: str, p=()):
    arr = _dbl_array(p)
    _check(load().bssn_set_initial_data(ctypes.c_void_p(ctx), ID_KIND[kind], arr, len(p)))


def bssn_set_adm(ctx: int, host_adm: np.ndarray, t: float = 0.0):
    assert host_adm.dtype == np.float64 and host_adm.flags.c_contiguous
    _check(load().bssn_set_adm(ctypes.c_void_p(ctx), ctypes.c_void_p(host_adm.ctypes.data), float(t)))


def bssn_set_punctures(ctx: int, punctures=()):
    flat = [float(v) for q in punctures for v in q]
    _check(load().bssn_set_punctures(ctypes.c_void_p(ctx), _dbl_array(flat), len(punctures)))


def bssn_track_punctures(ctx: int, enable: bool):
    _check(load().bssn_track_punctures(ctypes.c_void_p(ctx), 1 if enable else 0))


def bssn_get_punctures(ctx: int) -> np.ndarray:
    out = (ctypes.c_double * 32)()
    n = ctypes.c_int32()
    _check(load().bssn_get_punctures(ctypes.c_void_p(ctx), out, ctypes.byref(n)))
    return np.array(out[:4 * n.value], dtype=np.float64).reshape(n.value, 4)


def bssn_adm_integrals(ctx: int, d_dens=None) -> np.ndarray:
    out = (ctypes.c_double * 8)()
    _check(load().bssn_adm_integrals(ctypes.c_void_p(ctx), ctypes.c_void_p(d_dens or 0), out))
    return np.array(out[:], dtype=np.float64)


def bssn_set_matter(ctx: int, d_tmunu):
    _check(load().bssn_set_matter(ctypes.c_void_p(ctx), ctypes.c_void_p(d_tmunu or 0)))


def bssn_psi4(ctx: int, d_out: int):
    _check(load().bssn_psi4(ctypes.c_void_p(ctx), ctypes.c_void_p(d_out)))


def bssn_rhs(ctx: int, d_state, d_rhs: int):
    _check(load().bssn_rhs(ctypes.c_void_p(ctx), ctypes.c_void_p(d_state or 0), ctypes.c_void_p(d_rhs)))


def bssn_rk4_step(ctx: int, nsteps: int):
    _check(load().bssn_rk4_step(ctypes.c_void_p(ctx), int(nsteps)))


def bssn_constraints(ctx: int) -> np.ndarray:
    out = (ctypes.c_double * 16)()
    _check(load().bssn_constraints(ctypes.c_void_p(ctx), out))
    return np.array(out[:], dtype=np.float64)


def bssn_get_state(ctx: int, host: np.ndarray) -> float:
    assert host.dtype == np.float64 and host.flags.c_contiguous
    t = ctypes.c_double()
    _check(load().bssn_get_state(ctypes.c_void_p(ctx), ctypes.c_void_p(host.ctypes.data), ctypes.byref(t)))
    return t.value


def bssn_set_state(ctx: int, host: np.ndarray, t: float = 0.0):
    assert host.dtype == np.float64 and host.flags.c_contiguous
    _check(load().bssn_set_state(ctypes.c_void_p(ctx), ctypes.c_void_p(host.ctypes.data), float(t)))


def bssn_get_state_async(ctx: int, host: np.ndarray) -> float:
    """host: pinned, float64, C-contiguous; valid after bssn_wait_state."""
    assert host.dtype == np.float64 and host.flags.c_contiguous
    t = ctypes.c_double()
    _check(load().bssn_get_state_async(ctypes.c_void_p(ctx), ctypes.c_void_p(host.ctypes.data), ctypes.byref(t)))
    return t.value


def bssn_set_state_async(ctx: int, host: np.ndarray, t: float = 0.0):
    """host: pinned, float64, C-contiguous; unchanged until bssn_wait_state."""
    assert host.dtype == np.float64 and host.flags.c_contiguous
    _check(load().bssn_set_state_async(ctypes.c_void_p(ctx), ctypes.c_void_p(host.ctypes.data), float(t)))


def bssn_wait_state(ctx: int):
    _check(load().bssn_wait_state(ctypes.c_void_p(ctx)))


def bssn_tile_count() -> int:
    return int(load().bssn_tile_count())


def bssn_tile_name(cfg: int) -> str:
    return load().bssn_tile_name(int(cfg)).decode()


def bssn_set_tile(ctx: int, cfg: int):
    _check(load().bssn_set_tile(ctypes.c_void_p(ctx), int(cfg)))


def bssn_test_stall_tma(ctx: int, polls: int):
    """Test hook: TMA-staged stage kernels issue no copy and give up waiting
    after `polls` polls (0: normal operation); see include/bssn.h."""
    _check(load().bssn_test_stall_tma(ctypes.c_void_p(ctx), int(polls)))


def bssn_batch_test_stall_tma(batch: int, polls: int):
    """Test hook of the batch's TMA-staged stage kernel; see include/bssn.h."""
    _check(load().bssn_batch_test_stall_tma(ctypes.c_void_p(batch), int(polls)))


def bssn_autotune(ctx: int, reps: int = 3):
    """Time every tile configuration on the live state; selects and returns
    (best_index, {name: ms_per_launch})."""
    n = bssn_tile_count()
    ms = (ctypes.c_double * n)()
    best = ctypes.c_int32()
    _check(load().bssn_autotune(ctypes.c_void_p(ctx), int(reps), ctypes.byref(best), ms))
    return best.value, {bssn_tile_name(c): ms[c] for c in range(n)}


def bssn_profile(ctx: int, enable: bool):
    """Start (enable=True) or stop launch timing; on stop returns
    (stage_ms, stage_launches, boundary_ms, boundary_launches)."""
    out = (ctypes.c_double * 4)()
    _check(load().bssn_profile(ctypes.c_void_p(ctx), 1 if enable else 0, out))
    return None if enable else (out[0], int(out[1]), out[2], int(out[3]))


def bssn_serve_select(remaining_work, points, min_points: float) -> np.ndarray:
    """The shortest-work-first selection of the server on host arrays: a 0/1
    array marking the requests one step advances."""
    n = len(remaining_work)
    w = _dbl_array([float(v) for v in remaining_work])
    p = _dbl_array([float(v) for v in points])
    out = (ctypes.c_int32 * max(n, 1))()
    load().bssn_serve_select(int(n), w, p, float(min_points), out)
    return np.array(out[:n], dtype=np.int32)


def bssn_constraints_noalloc(params: Params, d_state: int, punctures=(), stream: int = 0) -> np.ndarray:
    """Constraint norms of a caller-held device state without a context and
    without any device allocation (see include/bssn.h)."""
    p = params.c()
    flat = [float(v) for q in punctures for v in q]
    arr = _dbl_array(flat)
    out = (ctypes.c_double * 16)()
    _check(load().bssn_constraints_noalloc(ctypes.byref(p), ctypes.c_void_p(d_state), arr,
                                           len(punctures), ctypes.c_void_p(stream), out))
    return np.array(out[:], dtype=np.float64)


def bssn_peak_probe(kind: str, d_sink: int, stream: int = 0, reps: int = 5) -> float:
    """Measured float64 ("fp64") or float32 ("fp32") fused multiply-add rate of
    the current GPU in GFLOP/s (see include/bssn.h); d_sink: >= 8 bytes of
    device memory."""
    out = ctypes.c_double()
    _check(load().bssn_peak_probe({"fp64": 0, "fp32": 1}[kind], ctypes.c_void_p(d_sink),
                                  ctypes.c_void_p(stream), int(reps), ctypes.byref(out)))
    return out.value


# ------------------------------------------------------- convenience class
class Evolution:
    """One evolution bound to a torch-owned device block and a CUDA stream."""

    def __init__(self, params: Params, device: str = "cuda", stream=None):
        import torch

        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU path)")
        self.params = params
        self.layout = bssn_layout_of(params)
        self.nbytes = bssn_required_bytes(params)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = bssn_alloc(params, self.mem.data_ptr(), self.nbytes, self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            bssn_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def enable_copy_staging(self):
        """Bind device staging areas (torch-owned) so that the asynchronous
        host copies overlap the steps (bssn_set_staging)."""
        p = self.params.c()
        n = int(load().bssn_staging_bytes(ctypes.byref(p)))
        if n == 0:
            raise BssnError(1, load().bssn_last_error().decode())
        self.staging = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        _check(load().bssn_set_staging(ctypes.c_void_p(self.ctx), ctypes.c_void_p(self.staging.data_ptr()), n))

    def disable_copy_staging(self):
        _check(load().bssn_set_staging(ctypes.c_void_p(self.ctx), None, 0))
        self.staging = None

    # register helpers (marshalling between host arrays and the padded layout)
    @property
    def shape(self):
        sx, sy, sz = self.layout["stored"]
        return (NUM_FIELDS, sz, sy, sx)

    def new_register(self):
        return self.torch.zeros(self.layout["register_elems"], dtype=self.torch.float64, device=self.device)

    def register_to_numpy(self, reg) -> np.ndarray:
        sx, sy, sz = self.layout["stored"]
        a = reg.view(NUM_FIELDS, sz, sy, self.layout["pitch"])[..., :sx]
        return a.cpu().numpy().copy()

    def numpy_to_register(self, arr: np.ndarray):
        sx, sy, sz = self.layout["stored"]
        reg = self.new_register()
        v = reg.view(NUM_FIELDS, sz, sy, self.layout["pitch"])
        v[..., :sx] = self.torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)).to(self.device)
        return reg

    def state_view(self):
        """torch view of y_n in the padded device layout (valid until the next step)."""
        sx, sy, sz = self.layout["stored"]
        ptr = bssn_state_ptr(self.ctx)
        off = (ptr - self.mem.data_ptr()) // 8
        flat = self.mem.view(self.torch.float64)
        return flat[off:off + self.layout["register_elems"]].view(NUM_FIELDS, sz, sy, self.layout["pitch"])

    # ABI calls
    def set_initial_data(self, kind, p=()):
        bssn_set_initial_data(self.ctx, kind, p)

    def rhs(self, state_reg=None):
        out = self.new_register()
        bssn_rhs(self.ctx, state_reg.data_ptr() if state_reg is not None else None, out.data_ptr())
        return out

    def rk4_step(self, nsteps=1):
        bssn_rk4_step(self.ctx, nsteps)

    def constraints(self):
        return bssn_constraints(self.ctx)

    def get_state(self):
        host = np.empty(self.shape, dtype=np.float64)
        t = bssn_get_state(self.ctx, host)
        return host, t

    def set_state(self, host: np.ndarray, t: float = 0.0):
        bssn_set_state(self.ctx, np.ascontiguousarray(host, dtype=np.float64), t)

    def set_adm(self, adm16: np.ndarray, t: float = 0.0):
        adm16 = np.ascontiguousarray(adm16, dtype=np.float64)
        assert adm16.shape == (16,) + self.shape[1:]
        bssn_set_adm(self.ctx, adm16, t)

    def set_punctures(self, punctures=()):
        bssn_set_punctures(self.ctx, punctures)

    def track_punctures(self, enable=True):
        bssn_track_punctures(self.ctx, enable)

    def get_punctures(self) -> np.ndarray:
        return bssn_get_punctures(self.ctx)

    def set_matter(self, tmunu=None):
        """Stress-energy tensor T_{mu nu}: a host array (10, Z, Y, X) in the order
        T_00, T_0x, T_0y, T_0z, T_xx, T_xy, T_xz, T_yy, T_yz, T_zz, copied to a
        device register this object keeps alive; None returns to vacuum."""
        if tmunu is None:
            bssn_set_matter(self.ctx, None)
            self._tmunu = None
            return
        sx, sy, sz = self.layout["stored"]
        t = np.ascontiguousarray(tmunu, dtype=np.float64)
        assert t.shape == (10, sz, sy, sx)
        reg = self.torch.zeros(10 * self.layout["field_stride"], dtype=self.torch.float64, device=self.device)
        reg.view(10, sz, sy, self.layout["pitch"])[..., :sx] = self.torch.from_numpy(t).to(self.device)
        self.torch.cuda.current_stream(self.device).synchronize()
        self._tmunu = reg
        bssn_set_matter(self.ctx, reg.data_ptr())

    def psi4(self, out=None):
        """Psi4 into a device register (2 * field_stride float64: real, then
        imaginary part, interior points); returns it (asynchronous)."""
        if out is None:
            out = self.torch.zeros(2 * self.layout["field_stride"], dtype=self.torch.float64, device=self.device)
        bssn_psi4(self.ctx, out.data_ptr())
        return out

    def psi4_to_numpy(self, reg) -> np.ndarray:
        sx, sy, sz = self.layout["stored"]
        return reg.view(2, sz, sy, self.layout["pitch"])[..., :sx].cpu().numpy().copy()

    def adm_integrals(self, densities=False):
        """(integrals8, dens): M, J_x, J_y, J_z over all interior points then
        over the excised set; dens (4, Z, Y, X) host copy of the integrands at
        interior points (zero elsewhere) when densities is true, else None."""
        if not densities:
            return bssn_adm_integrals(self.ctx), None
        sx, sy, sz = self.layout["stored"]
        fs = self.layout["field_stride"]
        reg = self.torch.zeros(4 * fs, dtype=self.torch.float64, device=self.device)
        out = bssn_adm_integrals(self.ctx, reg.data_ptr())
        d = reg.view(4, sz, sy, self.layout["pitch"])[..., :sx].cpu().numpy().copy()
        return out, d


# ---------------------------------------------------------------- batches
class Batch:
    """Many evolutions advanced together, one RK4 step per replay of a
    captured CUDA graph: by default each member's single-grid kernels in a
    launch chain of its own, the chains side by side; or one launch per RK4
    stage over every member's tiles (see include/bssn.h).  precision: "fp64",
    "mixed" or "ff".  Owns a torch device pool and a dedicated stream."""

    def __init__(self, precision: str = "fp64", pool_bytes: int = 1 << 30, max_members: int = 64,
                 device: str = "cuda"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(self.device)
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=self.device)
        self.precision = precision
        out = ctypes.c_void_p()
        torch.cuda.synchronize(self.device)
        _check(load().bssn_batch_create(PRECISION[precision], int(max_members),
                                        ctypes.c_void_p(self.pool.data_ptr()), int(pool_bytes),
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(out)))
        self.handle = out.value
        self.params = {}

    def close(self):
        if self.handle:
            _check(load().bssn_batch_free(ctypes.c_void_p(self.handle)))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def member_bytes(params: Params) -> int:
        p = params.c()
        n = load().bssn_batch_member_bytes(ctypes.byref(p))
        if n == 0:
            raise BssnError(1, load().bssn_last_error().decode())
        return int(n)

    def add(self, params: Params) -> int:
        p = params.c()
        mid = ctypes.c_int32()
        _check(load().bssn_batch_add(ctypes.c_void_p(self.handle), ctypes.byref(p), ctypes.byref(mid)))
        self.params[mid.value] = params
        return mid.value

    def remove(self, member: int):
        _check(load().bssn_batch_remove(ctypes.c_void_p(self.handle), int(member)))
        self.params.pop(member, None)

    def set_initial_data(self, member: int, kind: str, p=()):
        arr = _dbl_array(p)
        _check(load().bssn_batch_set_initial_data(ctypes.c_void_p(self.handle), int(member), ID_KIND[kind],
                                                  arr, len(p)))

    def _shape(self, member):
        lay = bssn_layout_of(self.params[member])
        sx, sy, sz = lay["stored"]
        return (NUM_FIELDS, sz, sy, sx)

    def set_state(self, member: int, host: np.ndarray, t: float = 0.0):
        host = np.ascontiguousarray(host, dtype=np.float64)
        assert host.shape == self._shape(member)
        _check(load().bssn_batch_set_state(ctypes.c_void_p(self.handle), int(member),
                                           ctypes.c_void_p(host.ctypes.data), float(t)))

    def get_state(self, member: int):
        host = np.empty(self._shape(member), dtype=np.float64)
        t = ctypes.c_double()
        _check(load().bssn_batch_get_state(ctypes.c_void_p(self.handle), int(member),
                                           ctypes.c_void_p(host.ctypes.data), ctypes.byref(t)))
        return host, t.value

    def step(self, nsteps: int = 1):
        _check(load().bssn_batch_step(ctypes.c_void_p(self.handle), int(nsteps)))

    def synchronize(self):
        self.stream.synchronize()

    def hold(self, member: int, hold: bool = True):
        """Keep the member resident but leave it out of the next steps (hold=False resumes it)."""
        _check(load().bssn_batch_hold(ctypes.c_void_p(self.handle), int(member), 1 if hold else 0))

    def constraints(self, member: int):
        out = (ctypes.c_double * 16)()
        _check(load().bssn_batch_constraints(ctypes.c_void_p(self.handle), int(member), out))
        return np.array(out[:])

    def set_tile(self, cfg: int):
        _check(load().bssn_batch_set_tile(ctypes.c_void_p(self.handle), int(cfg)))

    def autotune(self, reps: int = 2):
        n = int(load().bssn_batch_tile_count())
        ms = (ctypes.c_double * n)()
        best = ctypes.c_int32()
        _check(load().bssn_batch_autotune(ctypes.c_void_p(self.handle), int(reps), ctypes.byref(best), ms))
        names = [load().bssn_batch_tile_name(c).decode() for c in range(n)]
        return best.value, dict(zip(names, ms[:]))


class Server:
    """Continuous-batching server of evolution requests (C scheduler thread)."""

    def __init__(self, precision: str = "mixed", budget_bytes: int = 1 << 30, pool_bytes: int = None,
                 device: str = "cuda"):
        import torch
        self.torch = torch
        pool_bytes = int(pool_bytes or budget_bytes + (16 << 20))
        self.stream = torch.cuda.Stream(torch.device(device))
        self.pool = torch.empty(pool_bytes, dtype=torch.uint8, device=device)
        torch.cuda.synchronize()
        out = ctypes.c_void_p()
        _check(load().bssn_server_create(PRECISION[precision], int(budget_bytes),
                                         ctypes.c_void_p(self.pool.data_ptr()), pool_bytes,
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(out)))
        self.handle = out.value

    def submit(self, params: Params, kind: str, p=(), nsteps: int = 1) -> int:
        c = params.c()
        arr = _dbl_array(p)
        t = ctypes.c_uint64()
        _check(load().bssn_submit(ctypes.c_void_p(self.handle), ctypes.byref(c), ID_KIND[kind], arr, len(p),
                                  int(nsteps), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """None while pending; else (status, norms16, latency_s)."""
        norms = (ctypes.c_double * 16)()
        lat = ctypes.c_double()
        st = load().bssn_poll(ctypes.c_void_p(self.handle), ctypes.c_uint64(ticket), norms, ctypes.byref(lat))
        if st == 4:
            return None
        if st not in (0, 7):
            raise BssnError(st, load().bssn_last_error().decode())
        return st, np.array(norms[:]), lat.value

    def wait(self, ticket: int, timeout: float = 120.0):
        import time
        t0 = time.time()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.time() - t0 > timeout:
                raise TimeoutError(f"ticket {ticket} not done after {timeout} s")
            time.sleep(0.001)

    def detail(self, ticket: int):
        """For a finished request: (latency_s, queued_s, resident_s)."""
        out = (ctypes.c_double * 3)()
        st = load().bssn_poll_detail(ctypes.c_void_p(self.handle), ctypes.c_uint64(ticket), out)
        if st not in (0, 7):
            raise BssnError(st, load().bssn_last_error().decode())
        return out[0], out[1], out[2]

    def set_policy(self, policy: str = "all", min_points: float = 0.0):
        """Which resident requests a step advances: "all" (every one) or
        "shortest" (least remaining work first, until they hold min_points
        interior points)."""
        code = SERVE_POLICY[policy]
        _check(load().bssn_server_set_policy(ctypes.c_void_p(self.handle), code, float(min_points)))

    def stats(self):
        out = (ctypes.c_double * 8)()
        _check(load().bssn_server_stats(ctypes.c_void_p(self.handle), out))
        keys = ["completed", "failed", "queued", "resident", "point_updates", "busy_s", "wall_s", "bytes_used"]
        return dict(zip(keys, out[:]))

    def close(self):
        if self.handle:
            _check(load().bssn_server_destroy(ctypes.c_void_p(self.handle)))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
