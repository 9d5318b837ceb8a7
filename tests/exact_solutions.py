"""Exact vacuum spacetimes in 3+1 form, converted to BSSN variables, with their
exact time derivatives -- used to pin the oracle's right-hand side.

Nothing here uses the oracle or the CUDA library.  A spacetime is a 4-metric
g_{mu nu} in base coordinates, pulled back through a smooth, time-dependent
coordinate map (base coordinates as functions of the grid coordinates
(t, x, y, z)).  The ADM fields follow from g by the 3+1 split
(gamma_ij = g_ij, beta_i = g_0i, alpha^2 = beta^i beta_i - g_00), K_ij from
the ADM evolution equation for the metric,
    K_ij = (1 / 2 alpha) (-d_t gamma_ij + beta^k d_k gamma_ij
                          + gamma_kj d_i beta^k + gamma_ik d_j beta^k),
and the BSSN fields from the definitions of the paper's Sec. "Spacetime
Curvature Evolution" (phi = ln(det gamma)/12, W = exp(-2 phi), gt = e^{-4 phi}
gamma, K = gamma^ij K_ij, At = e^{-4 phi}(K_ij - gamma_ij K/3),
Gt^i = -d_j gt^{ij}).  All derivatives are exact: the whole chain is evaluated
in truncated Taylor arithmetic (tests/jets.py).

Because these are exact solutions of the vacuum Einstein equations, the BSSN
right-hand side of phi/W, gt, K, At and Gt evaluated on their data must equal
the exact time derivative up to the O(h^4) truncation error of the stencils,
whatever the gauge.  The gauge fields (alpha, beta, B) are checked against
their defining equations evaluated with exact values.
"""
from __future__ import annotations

import functools

import numpy as np

from jets import Jet, cos, sin, sqrt

SYM6 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
ETA = np.diag([-1.0, 1.0, 1.0, 1.0])


def minkowski(tb, xb):
    return [[ETA[a, b] for b in range(4)] for a in range(4)]


def kerr_schild(M):
    """Schwarzschild in Kerr-Schild form, g = eta + 2 (M/r) l l, l = (1, x/r)."""
    def g(tb, xb):
        r = sqrt(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2])
        H = r.recip() * M
        l = [1.0] + [xb[i] / r for i in range(3)]
        return [[(H * l[a] * l[b]) * 2.0 + ETA[a, b] for b in range(4)] for a in range(4)]
    return g


def _flat_wavy_map(t, x, y, z):
    e = 0.05
    tb = t + sin((x + 2.0 * y - z) * (2 * np.pi / 3) + t) * (e / 2)
    xb = [x + sin((y + z) * (2 * np.pi / 3) + t * 0.5) * e,
          y + cos((z - x) * (2 * np.pi / 3) - t) * (e / 2),
          z + sin((x - y) * (2 * np.pi / 3)) * cos(t) * (e / 2)]
    return tb, xb


def _flat_wavy_B(t, x, y, z):
    return [sin(x + 2.0 * z) * 0.1, cos(y - x) * 0.1, sin(x * y + z) * 0.1]


def _ks_wavy_map(t, x, y, z):
    e = 0.05
    xb = [x + sin(y - z + t * (1 / 3)) * e,
          y + cos(z + x) * (e / 2),
          z + sin(x + 2.0 * y - t * 0.5) * (e / 2)]
    return t, xb


def _ks_offset_map(t, x, y, z):
    e = 0.05
    xb = [x - 0.8 + sin(y + t * (1 / 3)) * e,
          y + 0.6 + cos(z - x) * (e / 2),
          z - 0.3 + sin(x + 2.0 * y - t * 0.5) * (e / 2)]
    return t, xb


def _ks_boost_map(t, x, y, z):
    # boosted slices (velocity 0.3 along x) of the displaced black hole
    v = 0.3
    gm = 1.0 / np.sqrt(1.0 - v * v)
    xs = x - 0.8 + sin(y + t * (1 / 3)) * 0.05
    return (t - xs * v) * gm, [(xs - t * v) * gm, y + 0.6, z - 0.3 + sin(x - y) * 0.025]


def _ks_wavy_B(t, x, y, z):
    return [cos(y + z) * 0.1, sin(z - x) * 0.1, cos(x + y) * 0.1]


def _gauge_wave_metric(A, d):
    """ds^2 = H (-dt^2 + dx^2) + dy^2 + dz^2, H = 1 - A sin(2 pi (x - t) / d):
    flat space in harmonic slicing with zero shift."""
    def g(tb, xb):
        H = 1.0 - sin((xb[0] - tb) * (2 * np.pi / d)) * A
        return [[-H, 0.0, 0.0, 0.0], [0.0, H, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]]
    return g


def _identity_map(t, x, y, z):
    return t, [x, y, z]


def _zero_B(t, x, y, z):
    return [x * 0.0, x * 0.0, x * 0.0]


def flrw(w, t0=1.0):
    """Spatially flat FLRW with a perfect fluid P = w rho:
    ds^2 = -dt^2 + a(t)^2 dx^2, a = (t/t0)^p, p = 2/(3(1+w)); returns the
    metric and the stress-energy tensor T_ab = (rho + P) u_a u_b + P g_ab with
    u = d_t, rho = 3 H^2/(8 pi), H = p/t (Friedmann's equations for G = 1)."""
    p = 2.0 / (3.0 * (1.0 + w))

    def a2(tb):
        return (tb * (1.0 / t0)) ** (2.0 * p)

    def metric(tb, xb):
        A = a2(tb)
        return [[-1.0, 0.0, 0.0, 0.0], [0.0, A, 0.0, 0.0], [0.0, 0.0, A, 0.0], [0.0, 0.0, 0.0, A]]

    def tmunu(tb, xb):
        H = tb.recip() * p
        rho = H * H * (3.0 / (8.0 * np.pi))
        P = rho * w
        A = a2(tb)
        z = tb * 0.0
        return [[rho, z, z, z], [z, P * A, z, z], [z, z, P * A, z], [z, z, z, P * A]]
    return metric, tmunu


def _flrw_wavy_map(t, x, y, z):
    # t0 + t with tilted, curved slices and a sheared, time-dependent grid
    e = 0.04
    tb = t + 1.0 + sin((x - 2.0 * y + z) * (2 * np.pi / 3) + t) * (e / 2)
    xb = [x + sin((y + z) * (2 * np.pi / 3) + t * 0.5) * e,
          y + cos((z - x) * (2 * np.pi / 3) - t) * (e / 2),
          z + sin((x - y) * (2 * np.pi / 3)) * cos(t) * (e / 2)]
    return tb, xb


SPACETIMES = {
    "gauge_wave": {"metric": _gauge_wave_metric(0.01, 1.0), "map": _identity_map, "B": _zero_B},
    # Flat space in a time-dependent, curl-carrying, anisotropic coordinate
    # system: curved slices (K != 0), non-trivial lapse and a shift whose
    # gradient is not symmetric.
    "flat_wavy": {"metric": minkowski, "map": _flat_wavy_map, "B": _flat_wavy_B},
    # Schwarzschild (M = 1) in Kerr-Schild form seen from a moving, sheared
    # grid: 3-curvature, conformal factor and Gt all non-trivial.
    "ks_wavy": {"metric": kerr_schild(1.0), "map": _ks_wavy_map, "B": _ks_wavy_B},
    # The same black hole displaced from the grid origin (and seen from a
    # wavy grid): radial lines from the origin are far from its principal
    # null directions, so the fiducial tetrad sees Psi4 of the size of Psi2.
    "ks_offset": {"metric": kerr_schild(1.0), "map": _ks_offset_map, "B": _ks_wavy_B},
    # Slices boosted against the Kerr-Schild ones: the normal observer is not
    # radial, so the magnetic part of the Weyl tensor (the Codazzi projection)
    # is non-zero, which no spherically symmetric slicing of Schwarzschild has.
    "ks_boost": {"metric": kerr_schild(1.0), "map": _ks_boost_map, "B": _ks_wavy_B},
    # Matter: dust and radiation FLRW universes seen from tilted, curved,
    # time-dependent coordinates (E, S, S_i and the trace-free S_ij all
    # non-zero on the slices).
    "flrw_dust": {"metric": flrw(0.0)[0], "tmunu": flrw(0.0)[1], "map": _flrw_wavy_map, "B": _flat_wavy_B},
    "flrw_rad": {"metric": flrw(1.0 / 3.0)[0], "tmunu": flrw(1.0 / 3.0)[1], "map": _flrw_wavy_map,
                 "B": _flat_wavy_B},
}


def _det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def _adj3(m):
    def c(i, j):  # cofactor C_ij
        r = [a for a in range(3) if a != i]
        s = [b for b in range(3) if b != j]
        v = m[r[0]][s[0]] * m[r[1]][s[1]] - m[r[0]][s[1]] * m[r[1]][s[0]]
        return v if (i + j) % 2 == 0 else -v
    return [[c(j, i) for j in range(3)] for i in range(3)]  # adjugate = C^T


def _four_metric(spec, X, Y, Z, time, want_jac=False):
    """Jets of the time, the grid coordinates and the 4-metric g_{mu nu} in
    grid coordinates (pulled back through the spacetime's coordinate map);
    with want_jac also the base coordinates and the Jacobian
    Jm[a][m] = d base^a / d x^m."""
    shape = X.shape
    T = Jet.var(0, np.full(shape, float(time)))
    xs = [Jet.var(1, X), Jet.var(2, Y), Jet.var(3, Z)]
    tb, xb = spec["map"](T, *xs)
    base = [tb] + list(xb)
    Jm = [[base[a].d(m) for m in range(4)] for a in range(4)]  # d base^a / d x^m
    gb = spec["metric"](tb, xb)
    g4 = [[None] * 4 for _ in range(4)]
    for m in range(4):
        for n in range(m, 4):
            s = None
            for a in range(4):
                for b in range(4):
                    gab = gb[a][b]
                    if not isinstance(gab, Jet) and gab == 0.0:
                        continue
                    term = Jm[a][m] * Jm[b][n] * gab
                    s = term if s is None else s + term
            g4[m][n] = g4[n][m] = s
    if want_jac:
        return T, xs, g4, tb, xb, Jm
    return T, xs, g4




def psi4_exact(name: str, X, Y, Z, time=0.0):
    """Psi4 = R_abcd n^a mb^b n^c mb^d from the exact 4-Riemann tensor (vacuum:
    Riemann = Weyl) of the spacetime in grid coordinates (t, x, y, z), with
    R^a_bcd = d_c G^a_bd - d_d G^a_bc + G^a_ce G^e_bd - G^a_de G^e_bc, and the
    fiducial tetrad in coordinate components: u^mu = (1, -beta^i)/alpha,
    n = (u - r)/sqrt2, mb = (theta - i phi)/sqrt2 with the triad (r, theta, phi)
    built from r = x^i, phi = (-y, x, 0), theta^i = sqrt(det g) g^ik eps_klm
    phi^l r^m and made orthonormal in gamma_ij in the order phi, r, theta.
    Nothing of the 3+1 split of the curvature is used."""
    spec = SPACETIMES[name]
    X, Y, Z = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (X, Y, Z)))
    _, _, g4 = _four_metric(spec, X, Y, Z, time)
    gam = [[g4[i + 1][j + 1] for j in range(3)] for i in range(3)]
    bl = [g4[0][i + 1] for i in range(3)]
    idet = _det3(gam).recip()
    gu = [[a * idet for a in row] for row in _adj3(gam)]
    bu = [gu[i][0] * bl[0] + gu[i][1] * bl[1] + gu[i][2] * bl[2] for i in range(3)]
    ia2 = (bu[0] * bl[0] + bu[1] * bl[1] + bu[2] * bl[2] - g4[0][0]).recip()  # 1 / alpha^2
    # inverse 4-metric from the 3+1 split
    ginv = [[None] * 4 for _ in range(4)]
    ginv[0][0] = -ia2
    for i in range(3):
        ginv[0][i + 1] = ginv[i + 1][0] = bu[i] * ia2
        for j in range(3):
            ginv[i + 1][j + 1] = gu[i][j] - bu[i] * bu[j] * ia2
    dg = [[[g4[a][b].d(m) for b in range(4)] for a in range(4)] for m in range(4)]  # dg[m][a][b]
    Gam = [[[None] * 4 for _ in range(4)] for _ in range(4)]
    for a in range(4):
        for b in range(4):
            for c in range(b, 4):
                acc = None
                for d in range(4):
                    t = ginv[a][d] * (dg[b][d][c] + dg[c][d][b] - dg[d][b][c]) * 0.5
                    acc = t if acc is None else acc + t
                Gam[a][b][c] = Gam[a][c][b] = acc
    G = np.array([[[Gam[a][b][c].val for c in range(4)] for b in range(4)] for a in range(4)])
    dG = np.array([[[[Gam[a][b][c].d(m).val for c in range(4)] for b in range(4)] for a in range(4)]
                   for m in range(4)])  # dG[m][a][b][c]
    Rup = (np.einsum("cabd...->abcd...", dG) - np.einsum("dabc...->abcd...", dG)
           + np.einsum("ace...,ebd...->abcd...", G, G) - np.einsum("ade...,ebc...->abcd...", G, G))
    g4v = np.array([[g4[a][b].val for b in range(4)] for a in range(4)])
    Rdn = np.einsum("ae...,ebcd...->abcd...", g4v, Rup)
    # tetrad
    gamv = g4v[1:, 1:]
    guv = np.array([[gu[i][j].val for j in range(3)] for i in range(3)])
    alpha = 1.0 / np.sqrt(ia2.val)
    beta = np.array([b.val for b in bu])
    rv = np.array([X, Y, Z])
    pv = np.array([-Y, X, np.zeros_like(X)])
    eps = np.zeros((3, 3, 3))
    for i, j, k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        eps[i, j, k], eps[j, i, k] = 1.0, -1.0
    sdet = np.sqrt(np.linalg.det(np.moveaxis(gamv, (0, 1), (-2, -1))))
    tv = sdet * np.einsum("ik...,klm,l...,m...->i...", guv, eps, pv, rv)

    def dot(u, v):
        return np.einsum("ij...,i...,j...->...", gamv, u, v)

    pv = pv / np.sqrt(dot(pv, pv))
    rv = rv - dot(rv, pv) * pv
    rv = rv / np.sqrt(dot(rv, rv))
    tv = tv - dot(tv, pv) * pv - dot(tv, rv) * rv
    tv = tv / np.sqrt(dot(tv, tv))
    s2 = 1.0 / np.sqrt(2.0)
    u4 = np.concatenate([(1.0 / alpha)[None], -beta / alpha])
    n4 = s2 * (u4 - np.concatenate([np.zeros_like(X)[None], rv]))
    mb4 = s2 * np.concatenate([np.zeros_like(X)[None], tv - 1j * pv])
    return np.einsum("abcd...,a...,b...,c...,d...->...", Rdn, n4, mb4, n4, mb4)


def evaluate(name: str, X, Y, Z, time=0.0, use_w=True):
    """Evaluate the spacetime on coordinate arrays.

    Returns (state, dtstate, grad):
      state  (24, ...) BSSN fields in the oracle's field order
      dtstate (24, ...) exact d_t of fields 0..16 (phi|W, gt, K, At, Gt);
              fields 17..23 are NaN (gauge: checked separately)
      grad dict with 'alpha' (3,...) d_k alpha, 'beta' (3,3,...) [i][k] = d_k beta^i,
              'Gt' (3,3,...) [i][k] = d_k Gt^i, 'B' (3,3,...) [i][k] = d_k B^i
    """
    spec = SPACETIMES[name]
    X, Y, Z = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (X, Y, Z)))
    shape = X.shape
    T, xs, g4, tb, xb, Jm = _four_metric(spec, X, Y, Z, time, want_jac=True)
    gam = [[g4[i + 1][j + 1] for j in range(3)] for i in range(3)]
    bl = [g4[0][i + 1] for i in range(3)]
    det = _det3(gam)
    idet = det.recip()
    gu = [[a * idet for a in row] for row in _adj3(gam)]
    bu = [gu[i][0] * bl[0] + gu[i][1] * bl[1] + gu[i][2] * bl[2] for i in range(3)]
    alpha = sqrt(bu[0] * bl[0] + bu[1] * bl[1] + bu[2] * bl[2] - g4[0][0])

    def dt(j):
        return j.d(0)

    def dx(j, k):
        return j.d(k + 1)

    Kij = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(i, 3):
            s = -dt(gam[i][j])
            for k in range(3):
                s = s + bu[k] * dx(gam[i][j], k) + gam[k][j] * dx(bu[k], i) + gam[i][k] * dx(bu[k], j)
            Kij[i][j] = Kij[j][i] = s / (alpha * 2.0)
    trK = None
    for i in range(3):
        for j in range(3):
            v = gu[i][j] * Kij[i][j]
            trK = v if trK is None else trK + v
    phi = det.log() * (1.0 / 12.0)
    W = det ** (-1.0 / 6.0)
    em4 = det ** (-1.0 / 3.0)
    gt = [gam[i][j] * em4 for (i, j) in SYM6]
    At = [(Kij[i][j] - gam[i][j] * trK * (1.0 / 3.0)) * em4 for (i, j) in SYM6]
    cbrt_det = det ** (1.0 / 3.0)
    gtu = [[gu[i][j] * cbrt_det for j in range(3)] for i in range(3)]
    Gt = [-(dx(gtu[i][0], 0) + dx(gtu[i][1], 1) + dx(gtu[i][2], 2)) for i in range(3)]
    Bv = spec["B"](T, *xs)

    chi = W if use_w else phi
    evolved = [chi] + gt + [trK] + At + Gt
    state = np.stack([f.val for f in evolved + [alpha] + bu + Bv])
    dts = np.full_like(state, np.nan)
    for f, j in enumerate(evolved):
        dts[f] = dt(j).val
    grad = {
        "dt_alpha": dt(alpha).val,
        "alpha": np.stack([dx(alpha, k).val for k in range(3)]),
        "beta": np.stack([np.stack([dx(bu[i], k).val for k in range(3)]) for i in range(3)]),
        "Gt": np.stack([np.stack([dx(Gt[i], k).val for k in range(3)]) for i in range(3)]),
        "B": np.stack([np.stack([dx(Bv[i], k).val for k in range(3)]) for i in range(3)]),
    }
    # Integrands of the ADM mass and angular momentum volume integrals: on
    # exact vacuum data the Hamiltonian and momentum constraints make them
    # divergences of the fluxes
    #   F^i   = -(1/2 pi) gt^ij d_j psi                       (M)
    #   G_i^l = (1/8 pi) eps_ijk x^j psi^6 gt^lm At_mk        (J_i)
    # with psi = e^{phi} = det(gamma)^{1/12}; the exact integrands are
    # d_i F^i and d_l G_i^l, and the box integrals are the outward fluxes.
    psi = det ** (1.0 / 12.0)
    psi6 = det ** 0.5
    Fm = [sum((gtu[i][j] * dx(psi, j) for j in range(3)), Jet.const(0.0, shape)) * (-1.0 / (2 * np.pi))
          for i in range(3)]
    At3 = [[At[SYM6.index((min(a, b), max(a, b)))] for b in range(3)] for a in range(3)]
    Amix = [[sum((gtu[l][m] * At3[m][k] for m in range(3)), Jet.const(0.0, shape)) for k in range(3)]
            for l in range(3)]
    G = [[Jet.const(0.0, shape) for _ in range(3)] for _ in range(3)]
    for i in range(3):
        for j in range(3):
            for k in range(3):
                eps = (i - j) * (j - k) * (k - i) / 2
                if eps == 0:
                    continue
                for l in range(3):
                    G[i][l] = G[i][l] + xs[j] * psi6 * Amix[l][k] * (eps / (8 * np.pi))
    grad["M_dens"] = sum(dx(Fm[i], i).val for i in range(3))
    grad["J_dens"] = np.stack([sum(dx(G[i][l], l).val for l in range(3)) for i in range(3)])
    grad["M_flux"] = np.stack([f.val for f in Fm])
    grad["J_flux"] = np.stack([np.stack([G[i][l].val for l in range(3)]) for i in range(3)])
    if "tmunu" in spec:
        # T_{mu nu} in grid coordinates: J^a_mu J^b_nu T_ab, rows T_00, T_0x,
        # T_0y, T_0z, T_xx, T_xy, T_xz, T_yy, T_yz, T_zz
        Tb = spec["tmunu"](tb, xb)
        order = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
        tm = []
        for (m, n) in order:
            acc = np.zeros(shape)
            for a in range(4):
                for b in range(4):
                    acc = acc + Jm[a][m].val * Jm[b][n].val * Tb[a][b].val
            tm.append(acc)
        grad["tmunu"] = np.stack(tm)
    grad["adm"] = np.stack([alpha.val] + [b.val for b in bu] +
                           [gam[i][j].val for (i, j) in SYM6] + [Kij[i][j].val for (i, j) in SYM6])
    return np.ascontiguousarray(state), dts, grad


@functools.lru_cache(maxsize=48)
def _on_grid_w(name, n, lo, hi):
    h = (hi - lo) / n[0]
    xs = [lo + (np.arange(n[d] + 6) - 3 + 0.5) * h for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return evaluate(name, X, Y, Z, use_w=True)


def on_grid(name, n, lo, hi, use_w=True):
    """evaluate() on the cell-centred grid of n = (n0, n1, n2) interior points
    with spacing (hi - lo)/n0 from xmin = (lo, lo, lo), three ghost layers;
    cached (the jets are the slow part of the pins), returned as copies.  The
    phi variant is derived from W: phi = -ln(W)/2, d_t phi = -d_t W / (2 W)."""
    st, dts, grad = _on_grid_w(name, tuple(n), float(lo), float(hi))
    st, dts = st.copy(), dts.copy()
    grad = {k: np.array(v, copy=True) for k, v in grad.items()}
    if not use_w:
        W = st[0].copy()
        st[0] = -0.5 * np.log(W)
        dts[0] = -0.5 * dts[0] / W
    return st, dts, grad
