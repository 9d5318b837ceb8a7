"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds no arithmetic of the method: it only draws reproducible random smooth
fields (low Fourier modes) with the value ranges a BSSN state needs (positive
W and lapse, positive-definite conformal metric), and the workload recipes
(grid, domain, puncture parameters) as plain numbers.  Random numbers are
passed to both the CUDA path and the oracle as inputs.
"""
from __future__ import annotations

import math

import numpy as np

NUM_FIELDS = 24
GHOST = 3


def grid_coords(n, xmin, h):
    """Coordinates of stored points per axis (cell-centred, 3 ghosts)."""
    return [xmin[d] + (np.arange(n[d] + 2 * GHOST) - GHOST + 0.5) * h for d in range(3)]


def smooth_field(rng, X, Y, Z, L, modes=3, amp=1.0):
    """Sum of a few random low-wavenumber sinusoids on a box of size L."""
    f = np.zeros(np.broadcast(X, Y, Z).shape)
    for _ in range(modes):
        k = rng.integers(-2, 3, size=3) * (2 * math.pi / L)
        ph = rng.uniform(0, 2 * math.pi)
        a = rng.uniform(-1, 1)
        f += a * np.sin(k[0] * X + k[1] * Y + k[2] * Z + ph)
    return amp * f / modes


def random_state(seed, n, xmin, h, amp=0.1, background=None):
    """A smooth random BSSN-shaped state on all stored points, (24, Z, Y, X).

    Every field gets a perturbation of relative size ``amp`` around a flat
    background (W = 1, gt = delta, alpha = 1) or around ``background`` if
    given, so that every term of the right-hand side is exercised."""
    rng = np.random.default_rng(seed)
    xs = grid_coords(n, xmin, h)
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    L = max(n) * h
    if background is None:
        st = np.zeros((NUM_FIELDS,) + X.shape)
        st[0] = 1.0
        st[1] = st[4] = st[6] = 1.0
        st[17] = 1.0
    else:
        st = np.array(background, dtype=np.float64, copy=True)
    for f in range(NUM_FIELDS):
        scale = amp * (1.0 if f in (0, 1, 4, 6, 17) else 0.5)
        p = smooth_field(rng, X, Y, Z, L, amp=scale)
        if f in (0, 17):  # keep W and alpha positive
            st[f] = st[f] * (1.0 + 0.5 * p)
        else:
            st[f] = st[f] + p
    return np.ascontiguousarray(st)


def random_tmunu(seed, n, xmin, h, amp=0.01):
    """A smooth random stress-energy tensor T_{mu nu} on all stored points,
    (10, Z, Y, X) in the order T_00, T_0x, T_0y, T_0z, T_xx, T_xy, T_xz, T_yy,
    T_yz, T_zz: a positive energy density amp (1 + 0.5 p) and momentum and
    stress components of size amp/2 (plain seeded numbers, no physics)."""
    rng = np.random.default_rng(seed)
    xs = grid_coords(n, xmin, h)
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    L = max(n) * h
    t = np.empty((10,) + X.shape)
    t[0] = amp * (1.0 + 0.5 * smooth_field(rng, X, Y, Z, L))
    for q in range(1, 10):
        t[q] = smooth_field(rng, X, Y, Z, L, amp=0.5 * amp)
    return np.ascontiguousarray(t)


# ---- workload recipes (plain numbers)
def single_puncture_128():
    """Brill-Lindquist M = 1 on [-8, 8]^3 at 128^3: the origin sits on a cell
    corner, half a cell from the nearest points in every direction."""
    return dict(n=(128, 128, 128), xmin=(-8.0, -8.0, -8.0), h=16.0 / 128, punctures=[(1.0, 0.0, 0.0, 0.0)])


def gauge_wave_24():
    return dict(n=(24, 24, 24), xmin=(-0.5, -0.5, -0.5), h=1.0 / 24, A=0.01, d=1.0)


def binary_bl_batch(seed=1111, count=64, sizes=(48, 64, 96, 128)):
    """Time-symmetric Brill-Lindquist binaries: masses U[0.3, 0.7], separation
    U[2, 6], punctures on the x-axis about the centre of mass, each snapped to
    the nearest cell face; domain [-L, L]^3 with L = max(8, 2 s) (m1 + m2)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m1, m2 = rng.uniform(0.3, 0.7, size=2)
        s = rng.uniform(2.0, 6.0)
        n = int(rng.choice(sizes))
        L = max(8.0, 2.0 * s) * (m1 + m2)
        h = 2 * L / n
        x1, x2 = s * m2 / (m1 + m2), -s * m1 / (m1 + m2)
        # cell faces sit at -L + j h
        x1 = -L + round((x1 + L) / h) * h
        x2 = -L + round((x2 + L) / h) * h
        out.append(dict(n=(n, n, n), xmin=(-L, -L, -L), h=h,
                        punctures=[(m1, x1, 0.0, 0.0), (m2, x2, 0.0, 0.0)]))
    return out
