/*
 * bssn_rhs.h -- the oracle's point-wise BSSN right-hand side (Sec. "Spacetime
 * Curvature Evolution") and Sommerfeld boundary right-hand side (Sec.
 * "Boundary Conditions"), with the grid description and the stencils they
 * use.
 *
 * TEST INFRASTRUCTURE ONLY, part of the oracle (see bssn_oracle.c): nothing of
 * the CUDA library includes it.
 *
 * Every arithmetic value is of type `real`, which the including file defines
 * before including this header:
 *  - bssn_oracle.c (C, the oracle proper): typedef double real -- plain
 *    IEEE float64, and the (real) casts below are no-ops;
 *  - bssn_oracle_instrumented.cpp (C++): a class that carries, beside the
 *    same float64 value computed by the same operations in the same order,
 *    the magnitude of the expression evaluated on absolute values (the
 *    scale of its rounding error) and a count of the operations.
 * Grid coordinates, the configuration and the state arrays stay double.
 * Data are read from the state as double and become real on first use.
 */
#ifndef BSSN_ORACLE_RHS_H
#define BSSN_ORACLE_RHS_H

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#define NF 24
#define GH 3

enum { F_CHI = 0, F_GT = 1, F_TRK = 7, F_AT = 8, F_GAM = 14, F_ALP = 17, F_BETA = 18, F_B = 21 };
enum { SL_1PLUSLOG = 0, SL_HARMONIC = 1, SL_GEODESIC = 2 };
enum { SH_GAMMA_DRIVER = 0, SH_FROZEN = 1 };
enum { ID_FLAT = 0, ID_GAUGE_WAVE = 1, ID_BL = 2, ID_KASNER = 3 };

/* Symmetric 3x3 component index -> storage offset (xx xy xz yy yz zz). */
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

typedef struct {
  int n[3];          /* interior points per axis */
  double xmin[3];    /* lower edge of the interior cell block */
  double h;          /* grid spacing, equal on all axes */
  int periodic;      /* 1: periodic ghosts; 0: Sommerfeld outer boundary */
  int use_w;         /* 1: evolve W = exp(-2 phi); 0: evolve phi */
  int slicing;       /* SL_* */
  int shift;         /* SH_* */
  double eta;        /* Gamma-driver damping constant */
  double q_R;        /* q(r) transition radius; <= 0 or inf -> q = 1 */
  double ko_eps;     /* Kreiss-Oliger epsilon */
  double dt;         /* RK4 time step */
  double w_floor;    /* lower bound on W wherever W is a divisor */
  double r_excise;   /* constraint-norm excision radius around punctures */
  int npunct;        /* punctures (for excision) */
  double punct[8][4];/* m, x, y, z */
  const double* tmunu; /* NULL (vacuum) or T_{mu nu}, 10 grids: T_00, T_0x,
                          T_0y, T_0z, T_xx, T_xy, T_xz, T_yy, T_yz, T_zz */
} ocfg;

/* ------------------------------------------------------------------ grid */

static inline int dimx(const ocfg* c, int d) { return c->n[d] + 2 * GH; }
static inline size_t npts(const ocfg* c) {
  return (size_t)dimx(c, 0) * dimx(c, 1) * dimx(c, 2);
}
static inline size_t pidx(const ocfg* c, int i, int j, int k) {
  return ((size_t)k * dimx(c, 1) + j) * dimx(c, 0) + i;
}
static inline double coord(const ocfg* c, int d, int i) {
  return c->xmin[d] + (i - GH + 0.5) * c->h;
}
static inline int is_interior(const ocfg* c, int i, int j, int k) {
  return i >= GH && i < GH + c->n[0] && j >= GH && j < GH + c->n[1] &&
         k >= GH && k < GH + c->n[2];
}


/* ------------------------------------------------------------ stencils
 * Sec. "Spacetime Curvature Evolution": fourth-order accurate finite
 * differences for the spacetime variables plus fifth-order Kreiss-Oliger
 * dissipation.  The coefficients are the standard ones (reading R1):
 *   D1  = (f-2 - 8 f-1 + 8 f1 - f2) / (12 h)
 *   D2  = (-f-2 + 16 f-1 - 30 f0 + 16 f1 - f2) / (12 h^2)
 *   Dxy = D1_x applied to D1_y
 *   upwind (beta >= 0): (-3 f-1 - 10 f0 + 18 f1 - 6 f2 + f3) / (12 h),
 *   mirrored for beta < 0
 *   KO  = +(eps / (64 h)) sum_d (f-3 - 6 f-2 + 15 f-1 - 20 f0 + 15 f1 - 6 f2 + f3)
 */
static const real C_D1[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
static const real C_D2[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
static const real C_UP[5] = {-3.0, -10.0, 18.0, -6.0, 1.0};
static const real C_KO[7] = {1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0};

static real st_d1(const double* p, ptrdiff_t s, double h) {
  real a = 0.0;
  for (int m = 0; m < 5; m++) a += C_D1[m] * p[(m - 2) * s];
  return a / (12.0 * h);
}
static real st_d2(const double* p, ptrdiff_t s, double h) {
  real a = 0.0;
  for (int m = 0; m < 5; m++) a += C_D2[m] * p[(m - 2) * s];
  return a / (12.0 * h * h);
}
static real st_d2m(const double* p, ptrdiff_t sa, ptrdiff_t sb, double h) {
  real a = 0.0;
  for (int m = 0; m < 5; m++)
    for (int q = 0; q < 5; q++) a += C_D1[m] * C_D1[q] * p[(m - 2) * sa + (q - 2) * sb];
  return a / (144.0 * h * h);
}
static real st_up(const double* p, ptrdiff_t s, double h, real b) {
  real a = 0.0;
  if (b >= 0.0) {
    for (int m = 0; m < 5; m++) a += C_UP[m] * p[(m - 1) * s];
  } else {
    for (int m = 0; m < 5; m++) a -= C_UP[m] * p[-(m - 1) * s];
  }
  return a / (12.0 * h);
}
static real st_ko(const double* p, ptrdiff_t s) {
  real a = 0.0;
  for (int m = 0; m < 7; m++) a += C_KO[m] * p[(m - 3) * s];
  return a;
}

/* Second derivative d_a d_b with a <= b or a > b: pure or mixed stencil. */
static real st_dd(const double* p, const ptrdiff_t str[3], int a, int b, double h) {
  if (a == b) return st_d2(p, str[a], h);
  return st_d2m(p, str[a], str[b], h);
}

/* ------------------------------------------------------- linear algebra */

static real det3(const real g[3][3]) {
  return g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
         g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
         g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
}
/* Matrix inverse by cofactors (no assumption det = 1). */
static void inv3(const real g[3][3], real gu[3][3]) {
  real d = det3(g);
  gu[0][0] = (g[1][1] * g[2][2] - g[1][2] * g[2][1]) / d;
  gu[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / d;
  gu[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / d;
  gu[1][0] = (g[1][2] * g[2][0] - g[1][0] * g[2][2]) / d;
  gu[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / d;
  gu[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / d;
  gu[2][0] = (g[1][0] * g[2][1] - g[1][1] * g[2][0]) / d;
  gu[2][1] = (g[0][1] * g[2][0] - g[0][0] * g[2][1]) / d;
  gu[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / d;
}

/* ------------------------------------------------------ matter sources
 * Sec. "Spacetime Curvature Evolution", the projections of the
 * stress-energy tensor T_{mu nu} (Sec. "TmunuBase") on the slice:
 *   E   = (T_00 - 2 beta^i T_0i + beta^i beta^j T_ij) / alpha^2
 *   S_i = -(T_0i - beta^j T_ij) / alpha
 *   S_ij = T_ij,  S = gamma^ij S_ij
 * (the printed T^{ij} in E is read as T_ij: E = n^mu n^nu T_{mu nu} with
 * n^mu = (1, -beta^i)/alpha).  gu_phys is gamma^ij. */
static void matter_projections(const ocfg* c, size_t id, real alpha, const real beta[3],
                               const real gu_phys[3][3], real* E, real Si[3],
                               real Sij[3][3], real* S) {
  const size_t S_ = npts(c);
  const double* T = c->tmunu;
  real T00 = T[id], T0[3], Tij[3][3];
  for (int a = 0; a < 3; a++) T0[a] = T[(size_t)(1 + a) * S_ + id];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) Tij[a][b] = T[(size_t)(4 + SYM[a][b]) * S_ + id];
  real e = T00;
  for (int a = 0; a < 3; a++) e -= 2.0 * beta[a] * T0[a];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) e += beta[a] * beta[b] * Tij[a][b];
  *E = e / (alpha * alpha);
  for (int a = 0; a < 3; a++) {
    real s = T0[a];
    for (int b = 0; b < 3; b++) s -= beta[b] * Tij[b][a];
    Si[a] = -s / alpha;
  }
  real tr = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      Sij[a][b] = Tij[a][b];
      tr += gu_phys[a][b] * Tij[a][b];
    }
  *S = tr;
}

/* ------------------------------------------------------------ BSSN RHS
 * Interior right-hand side at one point, Sec. "Spacetime Curvature
 * Evolution", equations for d_0 alpha, K, beta, B, phi, gt, At, Gt with
 * m = 1 and vacuum (E = S = S_i = S_ij = 0), the Ricci pieces Rt_ij and
 * Rphi_ij, 1+log / harmonic / geodesic slicing and the Gamma-driver.
 *
 * Readings (each also listed in the design notes):
 *  - d_0 = d_t - beta^j d_j acts on every variable; beta^j d_j X is the
 *    upwinded stencil chosen by the sign of beta^j.
 *  - d_k gt^{kj} is evaluated as -gt^{ka} gt^{jb} d_k gt_ab from the metric
 *    stencils, in Rt_ij and in the Gt equation; only gt_k(i d_j) Gt^k uses the
 *    evolved Gt.
 *  - In the B equation, d_0 Gt^i is the Gt equation's right side without
 *    advection and dissipation; e^{-4 phi} H = 1 for H = e^{4 phi}.
 *  - The Gt bracket reads 2 alpha [ -(2/3) gt^{ij} d_j K + Gt^i_kl At^kl
 *    + 6 At^ij d_j phi ] (m = 1 removes the d_k At^ki term).
 *  - [X]^TF = X_ij - (1/3) gt_ij gt^kl X_kl.
 *  - eta^i = eta B^i q(r) with eta a parameter; q = 1 for r <= R, R/r beyond.
 *  - W variant: W = exp(-2 phi), so e^{-4 phi} = W^2, d_i phi = -d_i W / (2W),
 *    d_i d_j phi = -d_i d_j W / (2W) + d_i W d_j W / (2 W^2), and
 *    d_0 W = (W/3)(alpha K - d_k beta^k); W is floored at w_floor only where
 *    it divides.
 *  - Frozen shift: the beta and B right-hand sides are identically zero.
 *  - Matter (when T_{mu nu} is given): the printed source terms -alpha S,
 *    -alpha e^{-4 phi} Shat_ij and -S^i are read in the normalisation of
 *    Einstein's equations G = 8 pi T that the paper's ADM mass integrand
 *    (16 pi E) uses: d_0 K gets +4 pi alpha (E + S), d_0 At_ij gets
 *    -8 pi alpha e^{-4 phi} [S_ij]^TF, d_0 Gt^i gets -16 pi alpha gt^ij S_j
 *    (and so does the Gamma-driver through d_0 Gt^i).
 */
static double q_of_r(const ocfg* c, double r) {
  if (!(c->q_R > 0.0) || isinf(c->q_R)) return 1.0;
  return r <= c->q_R ? 1.0 : c->q_R / r;
}

static void rhs_interior_point(const ocfg* c, const double* st, int i, int j, int k,
                               real out[NF]) {
  const size_t S = npts(c);
  const size_t id = pidx(c, i, j, k);
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  const double h = c->h;
#define P(f) (st + (size_t)(f) * S + id)
#define V(f) (st[(size_t)(f) * S + id])

  /* --- point values --- */
  real chi = V(F_CHI);
  real g[3][3], A[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      g[a][b] = V(F_GT + SYM[a][b]);
      A[a][b] = V(F_AT + SYM[a][b]);
    }
  real trK = V(F_TRK);
  real alpha = V(F_ALP);
  real beta[3], Bv[3];
  for (int a = 0; a < 3; a++) {
    beta[a] = V(F_BETA + a);
    Bv[a] = V(F_B + a);
  }

  /* --- centred derivatives --- */
  real dg[3][3][3];      /* dg[k][a][b] = d_k gt_ab */
  real ddg[3][3][3][3];  /* ddg[k][l][a][b] = d_k d_l gt_ab */
  real dchi[3], ddchi[3][3], dalp[3], ddalp[3][3], dK[3];
  real db[3][3];         /* db[k][a] = d_k beta^a */
  real ddb[3][3][3];     /* ddb[k][l][a] = d_k d_l beta^a */
  real dGt[3][3];        /* dGt[k][a] = d_k Gt^a */
  for (int kk = 0; kk < 3; kk++) {
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) dg[kk][a][b] = st_d1(P(F_GT + SYM[a][b]), str[kk], h);
    dchi[kk] = st_d1(P(F_CHI), str[kk], h);
    dalp[kk] = st_d1(P(F_ALP), str[kk], h);
    dK[kk] = st_d1(P(F_TRK), str[kk], h);
    for (int a = 0; a < 3; a++) {
      db[kk][a] = st_d1(P(F_BETA + a), str[kk], h);
      dGt[kk][a] = st_d1(P(F_GAM + a), str[kk], h);
    }
    for (int l = 0; l < 3; l++) {
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
          ddg[kk][l][a][b] = st_dd(P(F_GT + SYM[a][b]), str, kk, l, h);
      ddchi[kk][l] = st_dd(P(F_CHI), str, kk, l, h);
      ddalp[kk][l] = st_dd(P(F_ALP), str, kk, l, h);
      for (int a = 0; a < 3; a++) ddb[kk][l][a] = st_dd(P(F_BETA + a), str, kk, l, h);
    }
  }

  /* --- conformal factor: e^{-4 phi}, d phi, d d phi --- */
  real em4phi, dphi[3], ddphi[3][3];
  if (c->use_w) {
    real Wd = chi > c->w_floor ? chi : c->w_floor;
    em4phi = chi * chi;
    for (int a = 0; a < 3; a++) dphi[a] = -dchi[a] / (2.0 * Wd);
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++)
        ddphi[a][b] = -ddchi[a][b] / (2.0 * Wd) + dchi[a] * dchi[b] / (2.0 * Wd * Wd);
  } else {
    em4phi = exp(-4.0 * chi);
    for (int a = 0; a < 3; a++) dphi[a] = dchi[a];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) ddphi[a][b] = ddchi[a][b];
  }

  /* --- conformal geometry --- */
  real gu[3][3];
  inv3(g, gu);
  /* Christoffel symbols of the first kind, Gt_kij = (d_i g_kj + d_j g_ki - d_k g_ij)/2 */
  real G1[3][3][3];
  for (int kk = 0; kk < 3; kk++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++)
        G1[kk][a][b] = 0.5 * (dg[a][kk][b] + dg[b][kk][a] - dg[kk][a][b]);
  /* second kind, Gt^k_ij = gt^kl Gt_lij */
  real G2[3][3][3];
  for (int kk = 0; kk < 3; kk++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        real s = 0.0;
        for (int l = 0; l < 3; l++) s += gu[kk][l] * G1[l][a][b];
        G2[kk][a][b] = s;
      }
  /* dgu[k] = d_l gt^{lk} = -gt^{la} gt^{kb} d_l gt_ab */
  real dgu[3];
  for (int kk = 0; kk < 3; kk++) {
    real s = 0.0;
    for (int l = 0; l < 3; l++)
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) s -= gu[l][a] * gu[kk][b] * dg[l][a][b];
    dgu[kk] = s;
  }

  /* --- Rt_ij --- */
  real Rt[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      real s = 0.0;
      for (int kk = 0; kk < 3; kk++)
        for (int l = 0; l < 3; l++) s += -0.5 * gu[kk][l] * ddg[kk][l][a][b];
      for (int kk = 0; kk < 3; kk++)
        s += 0.5 * (g[kk][a] * dGt[b][kk] + g[kk][b] * dGt[a][kk]);
      for (int kk = 0; kk < 3; kk++)
        s -= 0.5 * (G1[a][b][kk] + G1[b][a][kk]) * dgu[kk];
      for (int l = 0; l < 3; l++)
        for (int m = 0; m < 3; m++) {
          real t = 0.0;
          for (int kk = 0; kk < 3; kk++)
            t += G2[kk][l][a] * G1[b][kk][m] + G2[kk][l][b] * G1[a][kk][m] +
                 G2[kk][a][m] * G1[kk][l][b];
          s += gu[l][m] * t;
        }
      Rt[a][b] = s;
    }

  /* --- Rphi_ij --- */
  real DDphi[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      real s = ddphi[a][b];
      for (int kk = 0; kk < 3; kk++) s -= G2[kk][a][b] * dphi[kk];
      DDphi[a][b] = s;
    }
  real lap_phi = 0.0, grad2_phi = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      lap_phi += gu[a][b] * DDphi[a][b];
      grad2_phi += gu[a][b] * dphi[a] * dphi[b];
    }
  real Rphi[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      Rphi[a][b] = -2.0 * DDphi[a][b] - 2.0 * g[a][b] * lap_phi + 4.0 * dphi[a] * dphi[b] -
                   4.0 * g[a][b] * grad2_phi;

  /* --- lapse second covariant derivative --- */
  real DDalp[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      real s = ddalp[a][b];
      for (int kk = 0; kk < 3; kk++) s -= G2[kk][a][b] * dalp[kk];
      DDalp[a][b] = s;
    }

  /* --- At with raised indices --- */
  real Auu[3][3], Aud[3][3];  /* At^ij, At^i_j */
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      real s = 0.0, t = 0.0;
      for (int kk = 0; kk < 3; kk++)
        for (int l = 0; l < 3; l++) s += gu[a][kk] * gu[b][l] * A[kk][l];
      for (int l = 0; l < 3; l++) t += gu[a][l] * A[l][b];
      Auu[a][b] = s;
      Aud[a][b] = t;
    }
  real AA = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) AA += Auu[a][b] * A[a][b];
  real divb = db[0][0] + db[1][1] + db[2][2];

  /* --- matter projections (zero in vacuum) --- */
  real Em = 0.0, Sm = 0.0, Smi[3] = {0.0, 0.0, 0.0}, Smij[3][3] = {{0.0}};
  if (c->tmunu) {
    real gphys[3][3];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) gphys[a][b] = em4phi * gu[a][b];
    matter_projections(c, id, alpha, beta, gphys, &Em, Smi, Smij, &Sm);
  }

  real r[NF];
  for (int f = 0; f < NF; f++) r[f] = 0.0;

  /* d_0 phi = -(alpha/6) K + (1/6) d_k beta^k ; W: d_0 W = (W/3)(alpha K - d_k beta^k) */
  if (c->use_w)
    r[F_CHI] = (chi / 3.0) * (alpha * trK - divb);
  else
    r[F_CHI] = -(alpha / 6.0) * trK + divb / 6.0;

  /* d_0 gt_ij = -2 alpha At_ij + 2 gt_k(i d_j) beta^k - (2/3) gt_ij d_k beta^k */
  for (int a = 0; a < 3; a++)
    for (int b = a; b < 3; b++) {
      real s = -2.0 * alpha * A[a][b];
      for (int kk = 0; kk < 3; kk++) s += g[kk][a] * db[b][kk] + g[kk][b] * db[a][kk];
      s -= (2.0 / 3.0) * g[a][b] * divb;
      r[F_GT + SYM[a][b]] = s;
    }

  /* d_0 K = -e^{-4phi}[Dt^i Dt_i alpha + 2 d_i phi Dt^i alpha] + alpha(At^ij At_ij + K^2/3) */
  {
    real lap_alp = 0.0, dphi_dalp = 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        lap_alp += gu[a][b] * DDalp[a][b];
        dphi_dalp += gu[a][b] * dphi[a] * dalp[b];
      }
    r[F_TRK] = -em4phi * (lap_alp + 2.0 * dphi_dalp) + alpha * (AA + trK * trK / 3.0) +
               4.0 * M_PI * alpha * (Em + Sm);
  }

  /* d_0 At_ij = e^{-4phi}[alpha Rt + alpha Rphi - DtDt alpha + 4 d_(i phi Dt_j) alpha]^TF
   *             + alpha K At_ij - 2 alpha At_ik At^k_j + 2 At_k(i d_j) beta^k
   *             - (2/3) At_ij d_k beta^k */
  {
    real X[3][3];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++)
        X[a][b] = alpha * Rt[a][b] + alpha * Rphi[a][b] - DDalp[a][b] +
                  2.0 * (dphi[a] * dalp[b] + dphi[b] * dalp[a]);
    real trX = 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) trX += gu[a][b] * X[a][b];
    for (int a = 0; a < 3; a++)
      for (int b = a; b < 3; b++) {
        real s = em4phi * (X[a][b] - g[a][b] * trX / 3.0);
        s += alpha * trK * A[a][b];
        for (int kk = 0; kk < 3; kk++) s -= 2.0 * alpha * A[a][kk] * Aud[kk][b];
        for (int kk = 0; kk < 3; kk++) s += A[kk][a] * db[b][kk] + A[kk][b] * db[a][kk];
        s -= (2.0 / 3.0) * A[a][b] * divb;
        if (c->tmunu) {
          /* [S_ij]^TF = S_ij - (1/3) gamma_ij S = S_ij - (1/3) gt_ij gt^kl S_kl */
          real trs = 0.0;
          for (int kk = 0; kk < 3; kk++)
            for (int l = 0; l < 3; l++) trs += gu[kk][l] * Smij[kk][l];
          s -= 8.0 * M_PI * alpha * em4phi * (Smij[a][b] - g[a][b] * trs / 3.0);
        }
        r[F_AT + SYM[a][b]] = s;
      }
  }

  /* d_0 Gt^i (without advection) */
  real gam_rhs[3];
  for (int a = 0; a < 3; a++) {
    real s = 0.0;
    for (int kk = 0; kk < 3; kk++)
      for (int l = 0; l < 3; l++) s += gu[kk][l] * ddb[kk][l][a];
    for (int jj = 0; jj < 3; jj++) {
      real ddiv = 0.0;
      for (int kk = 0; kk < 3; kk++) ddiv += ddb[jj][kk][kk];
      s += gu[a][jj] * ddiv / 3.0;
    }
    for (int jj = 0; jj < 3; jj++) s += dgu[jj] * db[jj][a];
    s -= (2.0 / 3.0) * dgu[a] * divb;
    for (int jj = 0; jj < 3; jj++) s -= 2.0 * Auu[a][jj] * dalp[jj];
    real br = 0.0;
    for (int jj = 0; jj < 3; jj++) br += -(2.0 / 3.0) * gu[a][jj] * dK[jj];
    for (int kk = 0; kk < 3; kk++)
      for (int l = 0; l < 3; l++) br += G2[a][kk][l] * Auu[kk][l];
    for (int jj = 0; jj < 3; jj++) br += 6.0 * Auu[a][jj] * dphi[jj];
    s += 2.0 * alpha * br;
    for (int jj = 0; jj < 3; jj++) s -= 16.0 * M_PI * alpha * gu[a][jj] * Smi[jj];
    gam_rhs[a] = s;
    r[F_GAM + a] = s;
  }

  /* lapse: d_0 alpha = -alpha^2 f (K - K0), K0 = 0; 1+log f = 2/alpha gives
   * -2 alpha K, harmonic f = 1 gives -alpha^2 K, geodesic f = 0 gives 0 */
  if (c->slicing == SL_1PLUSLOG)
    r[F_ALP] = -2.0 * alpha * trK;
  else if (c->slicing == SL_HARMONIC)
    r[F_ALP] = -alpha * alpha * trK;
  else
    r[F_ALP] = 0.0;

  /* shift: d_0 beta^i = alpha^2 G B^i with G = (3/4) alpha^-2, i.e. (3/4) B^i;
   * d_0 B^i = e^{-4phi} H d_0 Gt^i - eta B^i q(r) with H = e^{4 phi}, i.e.
   * d_0 Gt^i - eta q(r) B^i */
  if (c->shift == SH_GAMMA_DRIVER) {
    double x = coord(c, 0, i), y = coord(c, 1, j), z = coord(c, 2, k);
    double rr = sqrt(x * x + y * y + z * z);
    double q = q_of_r(c, rr);
    for (int a = 0; a < 3; a++) {
      r[F_BETA + a] = 0.75 * Bv[a];
      r[F_B + a] = gam_rhs[a] - c->eta * q * Bv[a];
    }
  }

  /* advection beta^j d_j X (upwinded) and Kreiss-Oliger dissipation, every field */
  for (int f = 0; f < NF; f++) {
    if (c->shift == SH_FROZEN && f >= F_BETA) {
      r[f] = 0.0;
      continue;
    }
    real adv = 0.0;
    for (int jj = 0; jj < 3; jj++) adv += beta[jj] * st_up(P(f), str[jj], h, beta[jj]);
    real ko = st_ko(P(f), str[0]) + st_ko(P(f), str[1]) + st_ko(P(f), str[2]);
    r[f] += adv + (c->ko_eps / (64.0 * h)) * ko;
  }
  for (int f = 0; f < NF; f++) out[f] = r[f];
#undef P
#undef V
}

/* ------------------------------------------------ Sommerfeld boundary
 * Sec. "Boundary Conditions": d_t X = -v^i d_i X - v0 (X - X0)/r with
 * v^i = v0 x^i / r, second-order derivatives (centred where both neighbours
 * are stored, one-sided inward otherwise), plus the power-law (p = 2)
 * correction, evaluated layer by layer from the innermost outwards.
 * Reading of the correction: with n the sum of the outward normals of the
 * faces the point lies beyond and j = b - n its inner neighbour,
 *   rhs_b = rad_b + (r_j / r_b)^p (rhs_j - rad_j),
 * where rhs_j is the already final right-hand side of the inner layer (or
 * interior).  X0 = 1 for alpha, W and the diagonal of gt, else 0; v0 = sqrt(2)
 * for alpha and K, else 1. */
static void sommerfeld_x0v0(const ocfg* c, int f, double* X0, double* v0) {
  *X0 = 0.0;
  *v0 = 1.0;
  if (f == F_ALP || (f == F_CHI && c->use_w) || f == F_GT + 0 || f == F_GT + 3 ||
      f == F_GT + 5)
    *X0 = 1.0;
  if (f == F_ALP || f == F_TRK) *v0 = sqrt(2.0);
}

static real rad_point(const ocfg* c, const double* st, int f, int i, int j, int k) {
  const size_t S = npts(c);
  const int I[3] = {i, j, k};
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  const double* p = st + (size_t)f * S + pidx(c, i, j, k);
  double x[3];
  for (int d = 0; d < 3; d++) x[d] = coord(c, d, I[d]);
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double X0, v0;
  sommerfeld_x0v0(c, f, &X0, &v0);
  real s = 0.0;
  for (int d = 0; d < 3; d++) {
    real der;
    ptrdiff_t sd = str[d];
    if (I[d] - 1 >= 0 && I[d] + 1 < dimx(c, d))
      der = ((real)p[sd] - p[-sd]) / (2.0 * c->h);
    else if (I[d] + 1 >= dimx(c, d))
      der = (3.0 * (real)p[0] - 4.0 * p[-sd] + p[-2 * sd]) / (2.0 * c->h);
    else
      der = -(3.0 * (real)p[0] - 4.0 * p[sd] + p[2 * sd]) / (2.0 * c->h);
    s += -v0 * (x[d] / r) * der;
  }
  return s - v0 * ((real)p[0] - X0) / r;
}

/* layer of a point: 0 interior, else max over axes of the distance beyond it */
static int layer_of(const ocfg* c, int i, int j, int k, int nrm[3]) {
  const int I[3] = {i, j, k};
  int L = 0;
  for (int d = 0; d < 3; d++) {
    int o = 0;
    nrm[d] = 0;
    if (I[d] < GH) {
      o = GH - I[d];
      nrm[d] = -1;
    } else if (I[d] >= GH + c->n[d]) {
      o = I[d] - (GH + c->n[d]) + 1;
      nrm[d] = 1;
    }
    if (o > L) L = o;
  }
  return L;
}

static double radius_at(const ocfg* c, int i, int j, int k) {
  double x = coord(c, 0, i), y = coord(c, 1, j), z = coord(c, 2, k);
  return sqrt(x * x + y * y + z * z);
}

/* RHS at a single stored point (interior or ghost), following the same
 * definition; ghosts recurse through their inner neighbour. */
static void rhs_at(const ocfg* c, const double* st, int i, int j, int k, real out[NF]) {
  int n[3];
  int L = layer_of(c, i, j, k, n);
  if (L == 0) {
    rhs_interior_point(c, st, i, j, k, out);
    return;
  }
  if (c->periodic) {
    for (int f = 0; f < NF; f++) out[f] = 0.0;
    return;
  }
  int ii = i - n[0], jj = j - n[1], kk = k - n[2];
  real inner[NF];
  rhs_at(c, st, ii, jj, kk, inner);
  double rb = radius_at(c, i, j, k), rj = radius_at(c, ii, jj, kk);
  double fac = (rj / rb) * (rj / rb);
  for (int f = 0; f < NF; f++) {
    if (c->shift == SH_FROZEN && f >= F_BETA) {
      out[f] = 0.0;
      continue;
    }
    out[f] = rad_point(c, st, f, i, j, k) + fac * (inner[f] - rad_point(c, st, f, ii, jj, kk));
  }
}

#endif /* BSSN_ORACLE_RHS_H */
