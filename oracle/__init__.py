"""CPU oracle for the BSSN moving-puncture hot path (TEST INFRASTRUCTURE ONLY).

A plain FP64 C statement of the discrete scheme of "The Einstein Toolkit"
(arXiv:1111.3344), Sec. "Spacetime Curvature Evolution" (BSSN equations,
Ricci pieces, gauge), Sec. "Initial Conditions", Sec. "Boundary Conditions"
(Sommerfeld/NewRad) and Sec. "Other analysis modules" (constraints).  The
arithmetic lives in ``bssn_oracle.c``; this module compiles it with gcc and
marshals numpy arrays through ctypes.

Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library shares no code with it.

Array convention: a state is a C-contiguous float64 array of shape
``(24, n2+6, n1+6, n0+6)`` -- field, z, y, x -- with three ghost layers on
every side and no padding.  Point index ``i`` on an axis sits at
``xmin + (i - 3 + 0.5) h``.

Parity status per function: every function is pinned by tests under
``tests/test_oracle_*.py``.  In the Sommerfeld condition, the pure
outgoing-wave part, the power-law correction (an exact C/r^2 tail carried
outwards), X0 (flat space stays exactly flat) and v0 = sqrt(2) for alpha and K
(the 1+log gauge speed) are pinned; v0 = 1 for the other fields is a reading
of an under-specified passage (parity unpinned for that choice).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

NF = 24
GHOST = 3

# field indices
F_CHI, F_GT, F_TRK, F_AT, F_GAM, F_ALP, F_BETA, F_B = 0, 1, 7, 8, 14, 17, 18, 21
FIELD_NAMES = (
    ["chi", "gt_xx", "gt_xy", "gt_xz", "gt_yy", "gt_yz", "gt_zz", "trK",
     "At_xx", "At_xy", "At_xz", "At_yy", "At_yz", "At_zz",
     "Gt_x", "Gt_y", "Gt_z", "alpha", "beta_x", "beta_y", "beta_z",
     "B_x", "B_y", "B_z"])

SLICING = {"1+log": 0, "harmonic": 1, "geodesic": 2}
SHIFT = {"gamma-driver": 0, "frozen": 1}
ID_KIND = {"flat": 0, "gauge_wave": 1, "bl": 2, "kasner": 3}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bssn_oracle.c")
_HDR = os.path.join(_HERE, "bssn_rhs.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_INSTR_SRC = os.path.join(_HERE, "bssn_oracle_instrumented.cpp")
_INSTR_PATH = os.path.join(_BUILD, "liboracle_instr.so")
_lock = threading.Lock()
_lib = None


class _OCfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("xmin", ctypes.c_double * 3),
        ("h", ctypes.c_double),
        ("periodic", ctypes.c_int),
        ("use_w", ctypes.c_int),
        ("slicing", ctypes.c_int),
        ("shift", ctypes.c_int),
        ("eta", ctypes.c_double),
        ("q_R", ctypes.c_double),
        ("ko_eps", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("w_floor", ctypes.c_double),
        ("r_excise", ctypes.c_double),
        ("npunct", ctypes.c_int),
        ("punct", (ctypes.c_double * 4) * 8),
        ("tmunu", ctypes.POINTER(ctypes.c_double)),
    ]


@dataclass
class Config:
    """Grid and method parameters (mirrors the C struct of the oracle)."""
    n: Sequence[int] = (24, 24, 24)
    xmin: Sequence[float] = (-0.5, -0.5, -0.5)
    h: float = 1.0 / 24.0
    periodic: bool = True
    use_w: bool = True
    slicing: str = "1+log"
    shift: str = "gamma-driver"
    eta: float = 2.0
    q_R: float = math.inf
    ko_eps: float = 0.1
    dt: float = 0.25 / 24.0
    w_floor: float = 1e-10
    r_excise: float = 1.0
    punctures: list = field(default_factory=list)  # [(m, x, y, z), ...]
    # stress-energy tensor T_{mu nu} (10, grid): T_00, T_0x, T_0y, T_0z, T_xx,
    # T_xy, T_xz, T_yy, T_yz, T_zz at every stored point; None = vacuum
    tmunu: Optional[np.ndarray] = None

    @property
    def shape(self):
        return (NF, self.n[2] + 2 * GHOST, self.n[1] + 2 * GHOST, self.n[0] + 2 * GHOST)

    def _c(self) -> _OCfg:
        c = _OCfg()
        for d in range(3):
            c.n[d] = int(self.n[d])
            c.xmin[d] = float(self.xmin[d])
        c.h = float(self.h)
        c.periodic = 1 if self.periodic else 0
        c.use_w = 1 if self.use_w else 0
        c.slicing = SLICING[self.slicing]
        c.shift = SHIFT[self.shift]
        c.eta = float(self.eta)
        c.q_R = float(self.q_R)
        c.ko_eps = float(self.ko_eps)
        c.dt = float(self.dt)
        c.w_floor = float(self.w_floor)
        c.r_excise = float(self.r_excise)
        if len(self.punctures) > 8:
            raise ValueError("at most 8 punctures")
        c.npunct = len(self.punctures)
        for a, p in enumerate(self.punctures):
            for q in range(4):
                c.punct[a][q] = float(p[q])
        if self.tmunu is not None:
            t = self.tmunu
            if not (isinstance(t, np.ndarray) and t.dtype == np.float64 and t.flags.c_contiguous
                    and t.shape == (10,) + self.shape[1:]):
                raise ValueError("tmunu must be a C-contiguous float64 array of shape (10, Z, Y, X)")
            c.tmunu = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return c

    def coords(self, axis: int) -> np.ndarray:
        i = np.arange(self.n[axis] + 2 * GHOST)
        return self.xmin[axis] + (i - GHOST + 0.5) * self.h


def _compile(out: str, cmd_tail, deps, force: bool) -> str:
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(q) for q in deps)):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.run([*cmd_tail[:1], *cmd_tail[1:], "-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile bssn_oracle.c with gcc into oracle/_build/liboracle.so, and the
    instrumented right-hand side (bssn_oracle_instrumented.cpp: magnitudes and
    operation counts of the same expressions) with g++ into
    oracle/_build/liboracle_instr.so."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        _compile(_LIB_PATH, ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                             "-std=gnu11", _SRC, "-lm"], (_SRC, _HDR), force)
        _compile(_INSTR_PATH, ["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-std=c++17", _INSTR_SRC], (_INSTR_SRC, _HDR), force)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    ip = P(ctypes.c_int)
    cp = P(_OCfg)
    lib.oracle_npoints.argtypes = [cp]
    lib.oracle_npoints.restype = ctypes.c_size_t
    lib.oracle_apply_stencil.argtypes = [cp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, dp, dp]
    lib.oracle_rhs.argtypes = [cp, dp, dp]
    lib.oracle_sommerfeld.argtypes = [cp, dp, dp]
    lib.oracle_rhs_points.argtypes = [cp, dp, ctypes.c_int, ip, dp]
    lib.oracle_fill_periodic.argtypes = [cp, dp]
    lib.oracle_rk4.argtypes = [cp, dp, ctypes.c_int]
    lib.oracle_rk4.restype = ctypes.c_int
    lib.oracle_initial_data.argtypes = [cp, ctypes.c_int, dp, ctypes.c_int, dp]
    lib.oracle_initial_data.restype = ctypes.c_int
    lib.oracle_adm_to_bssn.argtypes = [cp, dp, dp, dp, dp, dp]
    lib.oracle_extrapolate_ghosts.argtypes = [cp, dp]
    lib.oracle_adm_to_bssn_fd.argtypes = [cp, dp, dp]
    lib.oracle_adm_to_bssn_fd.restype = ctypes.c_int
    lib.oracle_constraints.argtypes = [cp, dp, dp, dp, dp]
    lib.oracle_constraints.restype = ctypes.c_int
    lib.oracle_constraints_points.argtypes = [cp, dp, ctypes.c_int, ip, dp]
    lib.oracle_constraints_points.restype = ctypes.c_int
    lib.oracle_adm_integrals.argtypes = [cp, dp, dp, dp]
    lib.oracle_adm_integrals.restype = ctypes.c_int
    lib.oracle_interp.argtypes = [cp, dp, dp]
    lib.oracle_interp.restype = ctypes.c_double
    lib.oracle_track_step.argtypes = [cp, dp, ctypes.c_int, dp, ctypes.c_double]
    lib.oracle_psi4.argtypes = [cp, dp, dp]
    lib.oracle_psi4.restype = ctypes.c_int
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(cfg: Config, st: np.ndarray) -> np.ndarray:
    st = np.ascontiguousarray(st, dtype=np.float64)
    if st.shape != cfg.shape:
        raise ValueError(f"state shape {st.shape} != {cfg.shape}")
    return st


def apply_stencil(cfg: Config, op: str, f: np.ndarray, a: int = 0, b: int = 0,
                  sign: float = 1.0) -> np.ndarray:
    """Apply one stencil to a scalar grid function (shape cfg.shape[1:])."""
    ops = {"d1": 0, "dd": 1, "up": 2, "ko": 3}
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == cfg.shape[1:]
    out = np.zeros_like(f)
    c = cfg._c()
    lib.oracle_apply_stencil(ctypes.byref(c), ops[op], a, b, float(sign), _dp(f), _dp(out))
    return out


def rhs(cfg: Config, st: np.ndarray) -> np.ndarray:
    """Right-hand side at every stored point (Sommerfeld ghosts, or 0 if periodic)."""
    lib = _load()
    st = _state(cfg, st)
    out = np.zeros_like(st)
    c = cfg._c()
    lib.oracle_rhs(ctypes.byref(c), _dp(st), _dp(out))
    return out


def sommerfeld(cfg: Config, st: np.ndarray, rhs_in: np.ndarray) -> np.ndarray:
    """Fill ghost-point right-hand sides by the Sommerfeld condition, given the
    interior right-hand side in rhs_in (returns a new array)."""
    lib = _load()
    st = _state(cfg, st)
    out = _state(cfg, rhs_in).copy()
    c = cfg._c()
    lib.oracle_sommerfeld(ctypes.byref(c), _dp(st), _dp(out))
    return out


def rhs_points(cfg: Config, st: np.ndarray, ijk: np.ndarray) -> np.ndarray:
    """Right-hand side at stored points ijk (shape (P, 3), x/y/z array indices)."""
    lib = _load()
    st = _state(cfg, st)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((ijk.shape[0], NF))
    c = cfg._c()
    lib.oracle_rhs_points(ctypes.byref(c), _dp(st), ijk.shape[0],
                          ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out))
    return out


_instr = None


def _load_instr():
    global _instr
    if _instr is None:
        _load()  # builds both libraries
        lib = ctypes.CDLL(_INSTR_PATH)
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        lib.oracle_rhs_points_mag.argtypes = [P(_OCfg), dp, ctypes.c_int, P(ctypes.c_int), dp, dp]
        lib.oracle_rhs_points_ext.argtypes = [P(_OCfg), dp, ctypes.c_int, P(ctypes.c_int), dp]
        lib.oracle_rhs_opcount.argtypes = [P(_OCfg), dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           P(ctypes.c_longlong)]
        _instr = lib
    return _instr


def rhs_points_mag(cfg: Config, st: np.ndarray, ijk: np.ndarray):
    """Right-hand side at stored points ijk (as rhs_points) by the instrumented
    build: (values, magnitudes), each (P, 24).  The values equal rhs_points
    bit for bit; a magnitude is the same expression evaluated on absolute
    values (every difference a sum), the scale that bounds the rounding error
    of any evaluation order of that expression (bssn_oracle_instrumented.cpp)."""
    lib = _load_instr()
    st = _state(cfg, st)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    val = np.zeros((ijk.shape[0], NF))
    mag = np.zeros((ijk.shape[0], NF))
    c = cfg._c()
    lib.oracle_rhs_points_mag(ctypes.byref(c), _dp(st), ijk.shape[0],
                              ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(val), _dp(mag))
    return val, mag


def rhs_mag(cfg: Config, st: np.ndarray):
    """rhs_points_mag at every stored point, as two arrays of the state's shape
    (24, Z, Y, X): the right-hand side (equal to rhs) and its magnitudes."""
    Z, Y, X = cfg.shape[1:]
    k, j, i = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    val, mag = rhs_points_mag(cfg, st, ijk)
    return (np.ascontiguousarray(val.T).reshape(cfg.shape), np.ascontiguousarray(mag.T).reshape(cfg.shape))


def rhs_points_ext(cfg: Config, st: np.ndarray, ijk: np.ndarray) -> np.ndarray:
    """The same right-hand side evaluated in long double (the instrumented
    build's second copy of the header), rounded to float64 at the end."""
    lib = _load_instr()
    st = _state(cfg, st)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((ijk.shape[0], NF))
    c = cfg._c()
    lib.oracle_rhs_points_ext(ctypes.byref(c), _dp(st), ijk.shape[0],
                              ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out))
    return out


def rhs_opcount(cfg: Config, st: np.ndarray, point) -> dict:
    """Operations of one right-hand-side evaluation (all 24 fields) at the
    stored point (i, j, k) in the oracle's printed arrangement: additions and
    subtractions, multiplications, divisions, square roots and exponentials."""
    lib = _load_instr()
    st = _state(cfg, st)
    out = (ctypes.c_longlong * 4)()
    c = cfg._c()
    i, j, k = (int(v) for v in point)
    lib.oracle_rhs_opcount(ctypes.byref(c), _dp(st), i, j, k, out)
    return {"add": out[0], "mul": out[1], "div": out[2], "fun": out[3]}


def fill_periodic(cfg: Config, st: np.ndarray) -> np.ndarray:
    lib = _load()
    st = _state(cfg, st).copy()
    c = cfg._c()
    lib.oracle_fill_periodic(ctypes.byref(c), _dp(st))
    return st


def rk4(cfg: Config, st: np.ndarray, nsteps: int) -> np.ndarray:
    """Advance nsteps classical RK4 steps; returns a new array."""
    lib = _load()
    y = _state(cfg, st).copy()
    c = cfg._c()
    if lib.oracle_rk4(ctypes.byref(c), _dp(y), int(nsteps)) != 0:
        raise MemoryError("oracle_rk4: allocation failed")
    return y


def initial_data(cfg: Config, kind: str, params: Sequence[float]) -> np.ndarray:
    """Analytic initial data converted to BSSN variables (all stored points)."""
    lib = _load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    st = np.zeros(cfg.shape)
    c = cfg._c()
    bad = lib.oracle_initial_data(ctypes.byref(c), ID_KIND[kind], _dp(p), p.size, _dp(st))
    if bad:
        raise ValueError(f"bad initial-data parameters for {kind}: {params}")
    return st


def adm_to_bssn(cfg: Config, alpha, beta3, gam6, K6) -> np.ndarray:
    """BSSN variables from ADM grids by the definitions (Gt and B set to 0)."""
    lib = _load()
    S = cfg.shape[1:]
    alpha = np.ascontiguousarray(alpha, dtype=np.float64).reshape(S)
    beta3 = np.ascontiguousarray(beta3, dtype=np.float64).reshape((3,) + S)
    gam6 = np.ascontiguousarray(gam6, dtype=np.float64).reshape((6,) + S)
    K6 = np.ascontiguousarray(K6, dtype=np.float64).reshape((6,) + S)
    st = np.zeros(cfg.shape)
    c = cfg._c()
    lib.oracle_adm_to_bssn(ctypes.byref(c), _dp(alpha), _dp(beta3), _dp(gam6), _dp(K6), _dp(st))
    return st


def extrapolate_ghosts(cfg: Config, f: np.ndarray) -> np.ndarray:
    """Cubic extrapolation of a scalar grid's ghost points from its interior."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    assert f.shape == cfg.shape[1:]
    c = cfg._c()
    lib.oracle_extrapolate_ghosts(ctypes.byref(c), _dp(f))
    return f


def adm_to_bssn_fd(cfg: Config, adm16: np.ndarray) -> np.ndarray:
    """BSSN state from ADM grids (16, Z, Y, X): alpha, beta^i, gamma_ij (6),
    K_ij (6); Gt^i by 4th-order differences inside, cubic extrapolation (or
    periodic copy) on the ghost layers, B^i = 0."""
    lib = _load()
    adm16 = np.ascontiguousarray(adm16, dtype=np.float64)
    assert adm16.shape == (16,) + cfg.shape[1:]
    st = np.zeros(cfg.shape)
    c = cfg._c()
    lib.oracle_adm_to_bssn_fd(ctypes.byref(c), _dp(adm16), _dp(st))
    return st


def constraints(cfg: Config, st: np.ndarray):
    """(norms16, H, M): norms in the order L2 H,Mx,My,Mz, Linf H,Mx,My,Mz,
    full interior then excised; H (grid) and M (3, grid) at interior points."""
    lib = _load()
    st = _state(cfg, st)
    out = np.zeros(16)
    H = np.zeros(cfg.shape[1:])
    M = np.zeros((3,) + cfg.shape[1:])
    c = cfg._c()
    if lib.oracle_constraints(ctypes.byref(c), _dp(st), _dp(out), _dp(H), _dp(M)) != 0:
        raise MemoryError("oracle_constraints: allocation failed")
    return out, H, M


def constraints_points(cfg: Config, st: np.ndarray, ijk: np.ndarray) -> np.ndarray:
    lib = _load()
    st = _state(cfg, st)
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    out = np.zeros((ijk.shape[0], 4))
    c = cfg._c()
    if lib.oracle_constraints_points(ctypes.byref(c), _dp(st), ijk.shape[0],
                                     ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     _dp(out)) != 0:
        raise MemoryError("oracle_constraints_points: allocation failed")
    return out


def adm_integrals(cfg: Config, st: np.ndarray):
    """(integrals8, dens): M, J_x, J_y, J_z as midpoint sums over all interior
    points, then over the points farther than r_excise from every puncture;
    dens (4, grid) holds the four integrands at interior points (0 elsewhere)."""
    lib = _load()
    st = _state(cfg, st)
    out = np.zeros(8)
    dens = np.zeros((4,) + cfg.shape[1:])
    c = cfg._c()
    lib.oracle_adm_integrals(ctypes.byref(c), _dp(st), _dp(out), _dp(dens))
    return out, dens


def interp(cfg: Config, f: np.ndarray, xyz) -> float:
    """Tricubic Lagrange interpolation of one grid function at a point."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == cfg.shape[1:]
    p = np.ascontiguousarray(xyz, dtype=np.float64)
    return lib.oracle_interp(ctypes.byref(cfg._c()), _dp(f), _dp(p))


def track_step(cfg: Config, st: np.ndarray, punctures, dt: float) -> np.ndarray:
    """One forward-Euler step of dx/dt = -beta at every puncture; punctures is
    (np, 4) rows {m, x, y, z}; returns the moved rows."""
    lib = _load()
    st = _state(cfg, st)
    pos = np.array(punctures, dtype=np.float64).reshape(-1, 4).copy()
    lib.oracle_track_step(ctypes.byref(cfg._c()), _dp(st), pos.shape[0], _dp(pos), float(dt))
    return pos


def psi4(cfg: Config, st: np.ndarray) -> np.ndarray:
    """Weyl scalar Psi4 (2, grid): real and imaginary parts at interior points
    (0 elsewhere)."""
    lib = _load()
    st = _state(cfg, st)
    out = np.zeros((2,) + cfg.shape[1:])
    if lib.oracle_psi4(ctypes.byref(cfg._c()), _dp(st), _dp(out)) != 0:
        raise MemoryError("oracle_psi4: allocation failed")
    return out
