/*
 * bssn_oracle.c -- plain FP64 CPU statement of the discrete BSSN
 * moving-puncture scheme of "The Einstein Toolkit" (arXiv:1111.3344),
 * Sec. "Spacetime Curvature Evolution" and its subsections.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA library
 * never calls, links or includes it, and it includes nothing of the CUDA
 * library: the two share no code, header, table or constant.
 *
 * Style: every quantity is written as the paper (or the stated reading of it)
 * defines it, with explicit index loops and no fusion, blocking or algebraic
 * rearrangement.  Build with -O2 -ffp-contract=off so that no multiply-add is
 * fused behind the reader's back.
 *
 * Storage: unpadded structure of arrays, st[f][k][j][i] with
 * i in [0, n0+6), j in [0, n1+6), k in [0, n2+6); ghost width 3.  Point
 * (i,j,k) sits at x = xmin + (i - 3 + 1/2) h (cell-centred grid).
 *
 * Field order (24 evolved grid functions, Sec. "Spacetime Curvature
 * Evolution": phi or W, the conformal metric, trK, the trace-free extrinsic
 * curvature, the conformal connection functions, lapse, shift and B^i):
 *   0 phi|W, 1..6 gt_xx gt_xy gt_xz gt_yy gt_yz gt_zz, 7 trK,
 *   8..13 At_xx .. At_zz, 14..16 Gt^x Gt^y Gt^z, 17 alpha, 18..20 beta^i,
 *   21..23 B^i.
 *
 * Parity pins (tests/test_oracle_*.py): stencil exactness on polynomials,
 * flat space staying flat, Kasner closed form under geodesic and 1+log
 * slicing, gauge-wave and boosted Kerr-Schild exact solutions at 4th order,
 * closed-form Hamiltonian/momentum constraints, Brill-Lindquist constraint
 * convergence, the outgoing-wave Sommerfeld condition.  The Sommerfeld
 * power-law correction term, the choice of X0/v0 per variable and the
 * initial lapse are readings of an under-specified passage: parity there is
 * unpinned beyond the pure-wave part.
 */
#include <complex.h>
#undef I /* the imaginary unit is written _Complex_I below */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

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

size_t oracle_npoints(const ocfg* c) { return npts(c); }

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
static const double C_D1[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
static const double C_D2[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
static const double C_UP[5] = {-3.0, -10.0, 18.0, -6.0, 1.0};
static const double C_KO[7] = {1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0};

static double st_d1(const double* p, ptrdiff_t s, double h) {
  double a = 0.0;
  for (int m = 0; m < 5; m++) a += C_D1[m] * p[(m - 2) * s];
  return a / (12.0 * h);
}
static double st_d2(const double* p, ptrdiff_t s, double h) {
  double a = 0.0;
  for (int m = 0; m < 5; m++) a += C_D2[m] * p[(m - 2) * s];
  return a / (12.0 * h * h);
}
static double st_d2m(const double* p, ptrdiff_t sa, ptrdiff_t sb, double h) {
  double a = 0.0;
  for (int m = 0; m < 5; m++)
    for (int q = 0; q < 5; q++) a += C_D1[m] * C_D1[q] * p[(m - 2) * sa + (q - 2) * sb];
  return a / (144.0 * h * h);
}
static double st_up(const double* p, ptrdiff_t s, double h, double b) {
  double a = 0.0;
  if (b >= 0.0) {
    for (int m = 0; m < 5; m++) a += C_UP[m] * p[(m - 1) * s];
  } else {
    for (int m = 0; m < 5; m++) a -= C_UP[m] * p[-(m - 1) * s];
  }
  return a / (12.0 * h);
}
static double st_ko(const double* p, ptrdiff_t s) {
  double a = 0.0;
  for (int m = 0; m < 7; m++) a += C_KO[m] * p[(m - 3) * s];
  return a;
}

/* Second derivative d_a d_b with a <= b or a > b: pure or mixed stencil. */
static double st_dd(const double* p, const ptrdiff_t str[3], int a, int b, double h) {
  if (a == b) return st_d2(p, str[a], h);
  return st_d2m(p, str[a], str[b], h);
}

/* Test hook: apply one stencil operator to a grid function at interior points.
 * op: 0 D1(a), 1 DD(a,b), 2 upwind(a, sign), 3 KO sum over all axes (no eps/64h).
 * Other points of out are set to 0. */
void oracle_apply_stencil(const ocfg* c, int op, int a, int b, double sign,
                          const double* f, double* out) {
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  memset(out, 0, npts(c) * sizeof(double));
  for (int k = GH; k < GH + c->n[2]; k++)
    for (int j = GH; j < GH + c->n[1]; j++)
      for (int i = GH; i < GH + c->n[0]; i++) {
        size_t id = pidx(c, i, j, k);
        const double* p = f + id;
        double v = 0.0;
        if (op == 0) v = st_d1(p, str[a], c->h);
        else if (op == 1) v = st_dd(p, str, a, b, c->h);
        else if (op == 2) v = st_up(p, str[a], c->h, sign);
        else if (op == 3) v = st_ko(p, 1) + st_ko(p, str[1]) + st_ko(p, str[2]);
        out[id] = v;
      }
}

/* ------------------------------------------------------- linear algebra */

static double det3(const double g[3][3]) {
  return g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
         g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
         g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
}
/* Matrix inverse by cofactors (no assumption det = 1). */
static void inv3(const double g[3][3], double gu[3][3]) {
  double d = det3(g);
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
static void matter_projections(const ocfg* c, size_t id, double alpha, const double beta[3],
                               const double gu_phys[3][3], double* E, double Si[3],
                               double Sij[3][3], double* S) {
  const size_t S_ = npts(c);
  const double* T = c->tmunu;
  double T00 = T[id], T0[3], Tij[3][3];
  for (int a = 0; a < 3; a++) T0[a] = T[(size_t)(1 + a) * S_ + id];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) Tij[a][b] = T[(size_t)(4 + SYM[a][b]) * S_ + id];
  double e = T00;
  for (int a = 0; a < 3; a++) e -= 2.0 * beta[a] * T0[a];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) e += beta[a] * beta[b] * Tij[a][b];
  *E = e / (alpha * alpha);
  for (int a = 0; a < 3; a++) {
    double s = T0[a];
    for (int b = 0; b < 3; b++) s -= beta[b] * Tij[b][a];
    Si[a] = -s / alpha;
  }
  double tr = 0.0;
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
                               double out[NF]) {
  const size_t S = npts(c);
  const size_t id = pidx(c, i, j, k);
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  const double h = c->h;
#define P(f) (st + (size_t)(f) * S + id)
#define V(f) (st[(size_t)(f) * S + id])

  /* --- point values --- */
  double chi = V(F_CHI);
  double g[3][3], A[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      g[a][b] = V(F_GT + SYM[a][b]);
      A[a][b] = V(F_AT + SYM[a][b]);
    }
  double trK = V(F_TRK);
  double alpha = V(F_ALP);
  double beta[3], Bv[3];
  for (int a = 0; a < 3; a++) {
    beta[a] = V(F_BETA + a);
    Bv[a] = V(F_B + a);
  }

  /* --- centred derivatives --- */
  double dg[3][3][3];      /* dg[k][a][b] = d_k gt_ab */
  double ddg[3][3][3][3];  /* ddg[k][l][a][b] = d_k d_l gt_ab */
  double dchi[3], ddchi[3][3], dalp[3], ddalp[3][3], dK[3];
  double db[3][3];         /* db[k][a] = d_k beta^a */
  double ddb[3][3][3];     /* ddb[k][l][a] = d_k d_l beta^a */
  double dGt[3][3];        /* dGt[k][a] = d_k Gt^a */
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
  double em4phi, dphi[3], ddphi[3][3];
  if (c->use_w) {
    double Wd = chi > c->w_floor ? chi : c->w_floor;
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
  double gu[3][3];
  inv3(g, gu);
  /* Christoffel symbols of the first kind, Gt_kij = (d_i g_kj + d_j g_ki - d_k g_ij)/2 */
  double G1[3][3][3];
  for (int kk = 0; kk < 3; kk++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++)
        G1[kk][a][b] = 0.5 * (dg[a][kk][b] + dg[b][kk][a] - dg[kk][a][b]);
  /* second kind, Gt^k_ij = gt^kl Gt_lij */
  double G2[3][3][3];
  for (int kk = 0; kk < 3; kk++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double s = 0.0;
        for (int l = 0; l < 3; l++) s += gu[kk][l] * G1[l][a][b];
        G2[kk][a][b] = s;
      }
  /* dgu[k] = d_l gt^{lk} = -gt^{la} gt^{kb} d_l gt_ab */
  double dgu[3];
  for (int kk = 0; kk < 3; kk++) {
    double s = 0.0;
    for (int l = 0; l < 3; l++)
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) s -= gu[l][a] * gu[kk][b] * dg[l][a][b];
    dgu[kk] = s;
  }

  /* --- Rt_ij --- */
  double Rt[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0;
      for (int kk = 0; kk < 3; kk++)
        for (int l = 0; l < 3; l++) s += -0.5 * gu[kk][l] * ddg[kk][l][a][b];
      for (int kk = 0; kk < 3; kk++)
        s += 0.5 * (g[kk][a] * dGt[b][kk] + g[kk][b] * dGt[a][kk]);
      for (int kk = 0; kk < 3; kk++)
        s -= 0.5 * (G1[a][b][kk] + G1[b][a][kk]) * dgu[kk];
      for (int l = 0; l < 3; l++)
        for (int m = 0; m < 3; m++) {
          double t = 0.0;
          for (int kk = 0; kk < 3; kk++)
            t += G2[kk][l][a] * G1[b][kk][m] + G2[kk][l][b] * G1[a][kk][m] +
                 G2[kk][a][m] * G1[kk][l][b];
          s += gu[l][m] * t;
        }
      Rt[a][b] = s;
    }

  /* --- Rphi_ij --- */
  double DDphi[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = ddphi[a][b];
      for (int kk = 0; kk < 3; kk++) s -= G2[kk][a][b] * dphi[kk];
      DDphi[a][b] = s;
    }
  double lap_phi = 0.0, grad2_phi = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      lap_phi += gu[a][b] * DDphi[a][b];
      grad2_phi += gu[a][b] * dphi[a] * dphi[b];
    }
  double Rphi[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      Rphi[a][b] = -2.0 * DDphi[a][b] - 2.0 * g[a][b] * lap_phi + 4.0 * dphi[a] * dphi[b] -
                   4.0 * g[a][b] * grad2_phi;

  /* --- lapse second covariant derivative --- */
  double DDalp[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = ddalp[a][b];
      for (int kk = 0; kk < 3; kk++) s -= G2[kk][a][b] * dalp[kk];
      DDalp[a][b] = s;
    }

  /* --- At with raised indices --- */
  double Auu[3][3], Aud[3][3];  /* At^ij, At^i_j */
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0, t = 0.0;
      for (int kk = 0; kk < 3; kk++)
        for (int l = 0; l < 3; l++) s += gu[a][kk] * gu[b][l] * A[kk][l];
      for (int l = 0; l < 3; l++) t += gu[a][l] * A[l][b];
      Auu[a][b] = s;
      Aud[a][b] = t;
    }
  double AA = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) AA += Auu[a][b] * A[a][b];
  double divb = db[0][0] + db[1][1] + db[2][2];

  /* --- matter projections (zero in vacuum) --- */
  double Em = 0.0, Sm = 0.0, Smi[3] = {0.0, 0.0, 0.0}, Smij[3][3] = {{0.0}};
  if (c->tmunu) {
    double gphys[3][3];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) gphys[a][b] = em4phi * gu[a][b];
    matter_projections(c, id, alpha, beta, gphys, &Em, Smi, Smij, &Sm);
  }

  double r[NF];
  for (int f = 0; f < NF; f++) r[f] = 0.0;

  /* d_0 phi = -(alpha/6) K + (1/6) d_k beta^k ; W: d_0 W = (W/3)(alpha K - d_k beta^k) */
  if (c->use_w)
    r[F_CHI] = (chi / 3.0) * (alpha * trK - divb);
  else
    r[F_CHI] = -(alpha / 6.0) * trK + divb / 6.0;

  /* d_0 gt_ij = -2 alpha At_ij + 2 gt_k(i d_j) beta^k - (2/3) gt_ij d_k beta^k */
  for (int a = 0; a < 3; a++)
    for (int b = a; b < 3; b++) {
      double s = -2.0 * alpha * A[a][b];
      for (int kk = 0; kk < 3; kk++) s += g[kk][a] * db[b][kk] + g[kk][b] * db[a][kk];
      s -= (2.0 / 3.0) * g[a][b] * divb;
      r[F_GT + SYM[a][b]] = s;
    }

  /* d_0 K = -e^{-4phi}[Dt^i Dt_i alpha + 2 d_i phi Dt^i alpha] + alpha(At^ij At_ij + K^2/3) */
  {
    double lap_alp = 0.0, dphi_dalp = 0.0;
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
    double X[3][3];
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++)
        X[a][b] = alpha * Rt[a][b] + alpha * Rphi[a][b] - DDalp[a][b] +
                  2.0 * (dphi[a] * dalp[b] + dphi[b] * dalp[a]);
    double trX = 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) trX += gu[a][b] * X[a][b];
    for (int a = 0; a < 3; a++)
      for (int b = a; b < 3; b++) {
        double s = em4phi * (X[a][b] - g[a][b] * trX / 3.0);
        s += alpha * trK * A[a][b];
        for (int kk = 0; kk < 3; kk++) s -= 2.0 * alpha * A[a][kk] * Aud[kk][b];
        for (int kk = 0; kk < 3; kk++) s += A[kk][a] * db[b][kk] + A[kk][b] * db[a][kk];
        s -= (2.0 / 3.0) * A[a][b] * divb;
        if (c->tmunu) {
          /* [S_ij]^TF = S_ij - (1/3) gamma_ij S = S_ij - (1/3) gt_ij gt^kl S_kl */
          double trs = 0.0;
          for (int kk = 0; kk < 3; kk++)
            for (int l = 0; l < 3; l++) trs += gu[kk][l] * Smij[kk][l];
          s -= 8.0 * M_PI * alpha * em4phi * (Smij[a][b] - g[a][b] * trs / 3.0);
        }
        r[F_AT + SYM[a][b]] = s;
      }
  }

  /* d_0 Gt^i (without advection) */
  double gam_rhs[3];
  for (int a = 0; a < 3; a++) {
    double s = 0.0;
    for (int kk = 0; kk < 3; kk++)
      for (int l = 0; l < 3; l++) s += gu[kk][l] * ddb[kk][l][a];
    for (int jj = 0; jj < 3; jj++) {
      double ddiv = 0.0;
      for (int kk = 0; kk < 3; kk++) ddiv += ddb[jj][kk][kk];
      s += gu[a][jj] * ddiv / 3.0;
    }
    for (int jj = 0; jj < 3; jj++) s += dgu[jj] * db[jj][a];
    s -= (2.0 / 3.0) * dgu[a] * divb;
    for (int jj = 0; jj < 3; jj++) s -= 2.0 * Auu[a][jj] * dalp[jj];
    double br = 0.0;
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
    double adv = 0.0;
    for (int jj = 0; jj < 3; jj++) adv += beta[jj] * st_up(P(f), str[jj], h, beta[jj]);
    double ko = st_ko(P(f), str[0]) + st_ko(P(f), str[1]) + st_ko(P(f), str[2]);
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

static double rad_point(const ocfg* c, const double* st, int f, int i, int j, int k) {
  const size_t S = npts(c);
  const int I[3] = {i, j, k};
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  const double* p = st + (size_t)f * S + pidx(c, i, j, k);
  double x[3];
  for (int d = 0; d < 3; d++) x[d] = coord(c, d, I[d]);
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double X0, v0;
  sommerfeld_x0v0(c, f, &X0, &v0);
  double s = 0.0;
  for (int d = 0; d < 3; d++) {
    double der;
    ptrdiff_t sd = str[d];
    if (I[d] - 1 >= 0 && I[d] + 1 < dimx(c, d))
      der = (p[sd] - p[-sd]) / (2.0 * c->h);
    else if (I[d] + 1 >= dimx(c, d))
      der = (3.0 * p[0] - 4.0 * p[-sd] + p[-2 * sd]) / (2.0 * c->h);
    else
      der = -(3.0 * p[0] - 4.0 * p[sd] + p[2 * sd]) / (2.0 * c->h);
    s += -v0 * (x[d] / r) * der;
  }
  return s - v0 * (p[0] - X0) / r;
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

/* ---------------------------------------------------------- full RHS */

void oracle_sommerfeld(const ocfg* c, const double* st, double* rhs);

/* rhs at every stored point: interior by the BSSN equations; ghost points by
 * the Sommerfeld condition (layers 1, 2, 3 in order) or 0 when periodic. */
void oracle_rhs(const ocfg* c, const double* st, double* rhs) {
  const size_t S = npts(c);
  memset(rhs, 0, (size_t)NF * S * sizeof(double));
#pragma omp parallel for schedule(dynamic)
  for (int k = GH; k < GH + c->n[2]; k++)
    for (int j = GH; j < GH + c->n[1]; j++)
      for (int i = GH; i < GH + c->n[0]; i++) {
        double o[NF];
        rhs_interior_point(c, st, i, j, k, o);
        size_t id = pidx(c, i, j, k);
        for (int f = 0; f < NF; f++) rhs[(size_t)f * S + id] = o[f];
      }
  if (c->periodic) return;
  oracle_sommerfeld(c, st, rhs);
}

/* Ghost-point right-hand sides by the Sommerfeld condition, layer 1, 2, 3 in
 * order, given the interior right-hand side already in rhs. */
void oracle_sommerfeld(const ocfg* c, const double* st, double* rhs) {
  const size_t S = npts(c);
  const int X = dimx(c, 0), Y = dimx(c, 1), Z = dimx(c, 2);
  for (int L = 1; L <= GH; L++) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < Z; k++)
      for (int j = 0; j < Y; j++)
        for (int i = 0; i < X; i++) {
          int n[3];
          if (layer_of(c, i, j, k, n) != L) continue;
          int ii = i - n[0], jj = j - n[1], kk = k - n[2];
          double rb = radius_at(c, i, j, k), rj = radius_at(c, ii, jj, kk);
          double fac = (rj / rb) * (rj / rb); /* p = 2 */
          size_t ib = pidx(c, i, j, k), ij = pidx(c, ii, jj, kk);
          for (int f = 0; f < NF; f++) {
            if (c->shift == SH_FROZEN && f >= F_BETA) continue;
            double radb = rad_point(c, st, f, i, j, k);
            double radj = rad_point(c, st, f, ii, jj, kk);
            rhs[(size_t)f * S + ib] = radb + fac * (rhs[(size_t)f * S + ij] - radj);
          }
        }
  }
}

/* RHS at a single stored point (interior or ghost), following the same
 * definition; ghosts recurse through their inner neighbour. */
static void rhs_at(const ocfg* c, const double* st, int i, int j, int k, double out[NF]) {
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
  double inner[NF];
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

/* RHS at a list of points ijk[3*p + d]; out[p*NF + f]. */
void oracle_rhs_points(const ocfg* c, const double* st, int np, const int* ijk, double* out) {
#pragma omp parallel for schedule(dynamic)
  for (int p = 0; p < np; p++) rhs_at(c, st, ijk[3 * p], ijk[3 * p + 1], ijk[3 * p + 2], out + (size_t)p * NF);
}

/* ------------------------------------------------------ periodic ghosts */
void oracle_fill_periodic(const ocfg* c, double* st) {
  const size_t S = npts(c);
  const int X = dimx(c, 0), Y = dimx(c, 1), Z = dimx(c, 2);
  for (int f = 0; f < NF; f++)
    for (int k = 0; k < Z; k++)
      for (int j = 0; j < Y; j++)
        for (int i = 0; i < X; i++) {
          if (is_interior(c, i, j, k)) continue;
          int si = GH + (((i - GH) % c->n[0]) + c->n[0]) % c->n[0];
          int sj = GH + (((j - GH) % c->n[1]) + c->n[1]) % c->n[1];
          int sk = GH + (((k - GH) % c->n[2]) + c->n[2]) % c->n[2];
          st[(size_t)f * S + pidx(c, i, j, k)] = st[(size_t)f * S + pidx(c, si, sj, sk)];
        }
}

/* ---------------------------------------------------------------- RK4
 * Method of lines with the classical fourth-order Runge-Kutta scheme:
 * k1 = f(y), k2 = f(y + dt k1/2), k3 = f(y + dt k2/2), k4 = f(y + dt k3),
 * y <- y + dt (k1 + 2 k2 + 2 k3 + k4) / 6.  The boundary right-hand side is
 * integrated like the interior; periodic ghosts are refreshed on every
 * stage state. */
int oracle_rk4(const ocfg* c, double* y, int nsteps) {
  const size_t M = (size_t)NF * npts(c);
  double* k1 = (double*)malloc(M * sizeof(double));
  double* k2 = (double*)malloc(M * sizeof(double));
  double* k3 = (double*)malloc(M * sizeof(double));
  double* k4 = (double*)malloc(M * sizeof(double));
  double* ys = (double*)malloc(M * sizeof(double));
  if (!k1 || !k2 || !k3 || !k4 || !ys) {
    free(k1); free(k2); free(k3); free(k4); free(ys);
    return 2;
  }
  const double dt = c->dt;
  for (int s = 0; s < nsteps; s++) {
    if (c->periodic) oracle_fill_periodic(c, y);
    oracle_rhs(c, y, k1);
    for (size_t q = 0; q < M; q++) ys[q] = y[q] + 0.5 * dt * k1[q];
    if (c->periodic) oracle_fill_periodic(c, ys);
    oracle_rhs(c, ys, k2);
    for (size_t q = 0; q < M; q++) ys[q] = y[q] + 0.5 * dt * k2[q];
    if (c->periodic) oracle_fill_periodic(c, ys);
    oracle_rhs(c, ys, k3);
    for (size_t q = 0; q < M; q++) ys[q] = y[q] + dt * k3[q];
    if (c->periodic) oracle_fill_periodic(c, ys);
    oracle_rhs(c, ys, k4);
    for (size_t q = 0; q < M; q++) y[q] = y[q] + dt * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]) / 6.0;
    if (c->periodic) oracle_fill_periodic(c, y);
  }
  free(k1); free(k2); free(k3); free(k4); free(ys);
  return 0;
}

/* ------------------------------------------------------- initial data
 * ADM data (alpha, beta, gamma_ij, K_ij) at a point, converted to BSSN by the
 * definitions of Sec. "Spacetime Curvature Evolution":
 *   phi = (1/12) ln det gamma (reading of the printed log[(1/12) det gamma];
 *   det gt = 1 fixes it), gt_ij = e^{-4 phi} gamma_ij, K = gamma^ij K_ij,
 *   At_ij = e^{-4 phi}(K_ij - gamma_ij K / 3), B^i = 0 (Sec. "Initial
 *   Conditions"), W = e^{-2 phi}.  Gt^i = -d_j gt^{ij} is taken in closed form
 *   for every data set here (it is zero except for the gauge wave).
 * kinds:
 *   FLAT: Minkowski.
 *   GAUGE_WAVE p = {A, d}: ds^2 = H(-dt^2 + dx^2) + dy^2 + dz^2 at t = 0,
 *     H = 1 - A sin(2 pi x / d); alpha = sqrt(H), gamma_xx = H,
 *     K_xx = H'/(2 sqrt H), Gt^x = (2/3) H' H^{-5/3}.
 *   BL p = {n, m1, x1, y1, z1, ...}: psi = 1 + sum m_a / (2 r_a),
 *     gamma = psi^4 delta, K_ij = 0 (the TwoPunctures decomposition with
 *     u = 1 at K = 0, Sec. "Initial Data"); alpha = psi^-2 (reading).
 *   KASNER p = {t0}: gamma = diag(t^{4/3}, t^{4/3}, t^{-2/3}),
 *     K_ij = -d_t gamma_ij / 2 = diag(-(2/3) t^{1/3}, -(2/3) t^{1/3},
 *     (1/3) t^{-5/3}), alpha = 1 (Sec. "Cosmology"). */
static int adm_point(int kind, const double* p, int np, const double x[3], double* alpha,
                     double beta[3], double gam[3][3], double Kij[3][3], double Gt[3]) {
  for (int a = 0; a < 3; a++) {
    beta[a] = 0.0;
    Gt[a] = 0.0;
    for (int b = 0; b < 3; b++) {
      gam[a][b] = (a == b) ? 1.0 : 0.0;
      Kij[a][b] = 0.0;
    }
  }
  *alpha = 1.0;
  if (kind == ID_FLAT) return 0;
  if (kind == ID_GAUGE_WAVE) {
    if (np < 2) return 1;
    double A = p[0], d = p[1];
    double H = 1.0 - A * sin(2.0 * M_PI * x[0] / d);
    double Hp = -A * (2.0 * M_PI / d) * cos(2.0 * M_PI * x[0] / d);
    *alpha = sqrt(H);
    gam[0][0] = H;
    Kij[0][0] = Hp / (2.0 * sqrt(H));
    Gt[0] = (2.0 / 3.0) * Hp * pow(H, -5.0 / 3.0);
    return 0;
  }
  if (kind == ID_BL) {
    if (np < 1) return 1;
    int n = (int)p[0];
    if (n < 1 || np < 1 + 4 * n) return 1;
    double psi = 1.0;
    for (int a = 0; a < n; a++) {
      const double* q = p + 1 + 4 * a;
      double dx = x[0] - q[1], dy = x[1] - q[2], dz = x[2] - q[3];
      psi += q[0] / (2.0 * sqrt(dx * dx + dy * dy + dz * dz));
    }
    double psi4 = psi * psi * psi * psi;
    for (int a = 0; a < 3; a++) gam[a][a] = psi4;
    *alpha = 1.0 / (psi * psi);
    return 0;
  }
  if (kind == ID_KASNER) {
    if (np < 1) return 1;
    double t = p[0];
    gam[0][0] = gam[1][1] = pow(t, 4.0 / 3.0);
    gam[2][2] = pow(t, -2.0 / 3.0);
    Kij[0][0] = Kij[1][1] = -(2.0 / 3.0) * pow(t, 1.0 / 3.0);
    Kij[2][2] = (1.0 / 3.0) * pow(t, -5.0 / 3.0);
    return 0;
  }
  return 1;
}

/* ADM -> BSSN by the definitions. */
static void adm_to_bssn(const ocfg* c, double alpha, const double beta[3],
                        const double gam[3][3], const double Kij[3][3], const double Gt[3],
                        double out[NF]) {
  double gu[3][3];
  inv3(gam, gu);
  double phi = log(det3(gam)) / 12.0;
  double em4 = exp(-4.0 * phi);
  double trK = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) trK += gu[a][b] * Kij[a][b];
  out[F_CHI] = c->use_w ? exp(-2.0 * phi) : phi;
  for (int a = 0; a < 3; a++)
    for (int b = a; b < 3; b++) {
      out[F_GT + SYM[a][b]] = em4 * gam[a][b];
      out[F_AT + SYM[a][b]] = em4 * (Kij[a][b] - gam[a][b] * trK / 3.0);
    }
  out[F_TRK] = trK;
  for (int a = 0; a < 3; a++) {
    out[F_GAM + a] = Gt[a];
    out[F_BETA + a] = beta[a];
    out[F_B + a] = 0.0;
  }
  out[F_ALP] = alpha;
}

int oracle_initial_data(const ocfg* c, int kind, const double* p, int np, double* st) {
  const size_t S = npts(c);
  const int X = dimx(c, 0), Y = dimx(c, 1), Z = dimx(c, 2);
  int bad = 0;
  for (int k = 0; k < Z; k++)
    for (int j = 0; j < Y; j++)
      for (int i = 0; i < X; i++) {
        double x[3] = {coord(c, 0, i), coord(c, 1, j), coord(c, 2, k)};
        double alpha, beta[3], gam[3][3], Kij[3][3], Gt[3], o[NF];
        if (adm_point(kind, p, np, x, &alpha, beta, gam, Kij, Gt)) bad = 1;
        adm_to_bssn(c, alpha, beta, gam, Kij, Gt, o);
        size_t id = pidx(c, i, j, k);
        for (int f = 0; f < NF; f++) st[(size_t)f * S + id] = o[f];
      }
  return bad;
}

/* General ADM -> BSSN on a whole grid (no derivatives): gam6/K6 in xx xy xz yy
 * yz zz order per point; Gt is set to 0 and must be supplied separately. */
void oracle_adm_to_bssn(const ocfg* c, const double* alpha, const double* beta3,
                        const double* gam6, const double* K6, double* st) {
  const size_t S = npts(c);
  for (size_t id = 0; id < S; id++) {
    double g[3][3], K[3][3], b[3], Gt[3] = {0, 0, 0}, o[NF];
    for (int a = 0; a < 3; a++)
      for (int bb = 0; bb < 3; bb++) {
        g[a][bb] = gam6[(size_t)SYM[a][bb] * S + id];
        K[a][bb] = K6[(size_t)SYM[a][bb] * S + id];
      }
    for (int a = 0; a < 3; a++) b[a] = beta3[(size_t)a * S + id];
    adm_to_bssn(c, alpha[id], b, g, K, Gt, o);
    for (int f = 0; f < NF; f++) st[(size_t)f * S + id] = o[f];
  }
}

/* ------------------------------------- ADM -> BSSN with Gt by differences
 * Sec. "Initial Conditions": the BSSN variables from their definitions, with
 * B^i = 0 and Gt^i = gt^{jk} Gt^i_jk from 4th-order first derivatives of gt_ij
 * at interior points, and cubic extrapolation of Gt^i at the outer boundary:
 * points on faces are extrapolated perpendicular to the face, points on edges
 * and corners along the sum of the adjoining faces' normals, layer by layer
 * from the innermost, each layer from the interior and the layers already set.
 * Reading: the extrapolation through the four points b - n, ..., b - 4n is the
 * cubic one, v(b) = 4 v(b-n) - 6 v(b-2n) + 4 v(b-3n) - v(b-4n). */

/* Cubic extrapolation of a scalar grid's ghost points from its interior. */
void oracle_extrapolate_ghosts(const ocfg* c, double* f) {
  const int X = dimx(c, 0), Y = dimx(c, 1), Z = dimx(c, 2);
  for (int L = 1; L <= GH; L++)
    for (int k = 0; k < Z; k++)
      for (int j = 0; j < Y; j++)
        for (int i = 0; i < X; i++) {
          int n[3];
          if (layer_of(c, i, j, k, n) != L) continue;
          double v[5];
          for (int m = 1; m <= 4; m++) v[m] = f[pidx(c, i - m * n[0], j - m * n[1], k - m * n[2])];
          f[pidx(c, i, j, k)] = 4.0 * v[1] - 6.0 * v[2] + 4.0 * v[3] - v[4];
        }
}

/* adm16[q][k][j][i]: q = alpha, beta^x, beta^y, beta^z, gamma_xx..zz (6), K_xx..zz (6). */
int oracle_adm_to_bssn_fd(const ocfg* c, const double* adm16, double* st) {
  const size_t S = npts(c);
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  for (size_t id = 0; id < S; id++) {
    double g[3][3], K[3][3], b[3], Gt[3] = {0, 0, 0}, o[NF];
    for (int a = 0; a < 3; a++)
      for (int bb = 0; bb < 3; bb++) {
        g[a][bb] = adm16[(size_t)(4 + SYM[a][bb]) * S + id];
        K[a][bb] = adm16[(size_t)(10 + SYM[a][bb]) * S + id];
      }
    for (int a = 0; a < 3; a++) b[a] = adm16[(size_t)(1 + a) * S + id];
    adm_to_bssn(c, adm16[id], b, g, K, Gt, o);
    for (int f = 0; f < NF; f++) st[(size_t)f * S + id] = o[f];
  }
  /* Gt^i = gt^{jk} gt^{il} Gt_ljk at interior points */
  for (int k = GH; k < GH + c->n[2]; k++)
    for (int j = GH; j < GH + c->n[1]; j++)
      for (int i = GH; i < GH + c->n[0]; i++) {
        size_t id = pidx(c, i, j, k);
        double g[3][3], gu[3][3], dg[3][3][3];
        for (int a = 0; a < 3; a++)
          for (int bb = 0; bb < 3; bb++) {
            const double* p = st + (size_t)(F_GT + SYM[a][bb]) * S + id;
            g[a][bb] = p[0];
            for (int d = 0; d < 3; d++) dg[d][a][bb] = st_d1(p, str[d], c->h);
          }
        inv3(g, gu);
        for (int a = 0; a < 3; a++) {
          double s = 0.0;
          for (int jj = 0; jj < 3; jj++)
            for (int kk = 0; kk < 3; kk++)
              for (int l = 0; l < 3; l++)
                s += gu[jj][kk] * gu[a][l] * 0.5 * (dg[jj][l][kk] + dg[kk][l][jj] - dg[l][jj][kk]);
          st[(size_t)(F_GAM + a) * S + id] = s;
        }
      }
  if (c->periodic) {
    oracle_fill_periodic(c, st);
  } else {
    for (int a = 0; a < 3; a++) oracle_extrapolate_ghosts(c, st + (size_t)(F_GAM + a) * S);
  }
  return 0;
}

/* -------------------------------------------------------- constraints
 * Sec. "Other analysis modules": H = R - K^i_j K^j_i + K^2 and
 * M_i = nabla_j K_i^j - nabla_i K (vacuum), from the ADM variables
 * gamma_ij = e^{4 phi} gt_ij and K_ij = e^{4 phi}(At_ij + gt_ij K / 3) formed
 * pointwise and then differenced with the 4th-order stencils.
 * R_ij = d_k Gamma^k_ij - d_j Gamma^k_ik + Gamma^k_kl Gamma^l_ij
 *        - Gamma^k_jl Gamma^l_ik, with d_m Gamma^k_ij from the chain rule
 *        (d_m gamma^kl = -gamma^ka gamma^lb d_m gamma_ab).
 * K in H is the trace gamma^ij K_ij of the ADM K_ij; M_i is written with
 * metric compatibility, gamma^jk (nabla_k K_ij - nabla_i K_jk). */
static void adm_grids(const ocfg* c, const double* st, double* gam6, double* K6) {
  const size_t S = npts(c);
  for (size_t id = 0; id < S; id++) {
    double chi = st[(size_t)F_CHI * S + id];
    double e4 = c->use_w ? 1.0 / (chi * chi) : exp(4.0 * chi);
    double trK = st[(size_t)F_TRK * S + id];
    for (int m = 0; m < 6; m++) {
      double g = st[(size_t)(F_GT + m) * S + id];
      gam6[(size_t)m * S + id] = e4 * g;
      K6[(size_t)m * S + id] = e4 * (st[(size_t)(F_AT + m) * S + id] + g * trK / 3.0);
    }
  }
}

static void constraints_point(const ocfg* c, const double* gam6, const double* K6, int i,
                              int j, int k, double out[4]) {
  const size_t S = npts(c);
  const size_t id = pidx(c, i, j, k);
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  const double h = c->h;
  double g[3][3], K[3][3], dg[3][3][3], ddg[3][3][3][3], dKd[3][3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      const double* pg = gam6 + (size_t)SYM[a][b] * S + id;
      const double* pk = K6 + (size_t)SYM[a][b] * S + id;
      g[a][b] = pg[0];
      K[a][b] = pk[0];
      for (int m = 0; m < 3; m++) {
        dg[m][a][b] = st_d1(pg, str[m], h);
        dKd[m][a][b] = st_d1(pk, str[m], h);
        for (int n = 0; n < 3; n++) ddg[m][n][a][b] = st_dd(pg, str, m, n, h);
      }
    }
  double gu[3][3];
  inv3(g, gu);
  /* Gamma_lij (first kind) and its derivative d_m Gamma_lij */
  double G1[3][3][3], dG1[3][3][3][3];
  for (int l = 0; l < 3; l++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        G1[l][a][b] = 0.5 * (dg[a][l][b] + dg[b][l][a] - dg[l][a][b]);
        for (int m = 0; m < 3; m++)
          dG1[m][l][a][b] = 0.5 * (ddg[m][a][l][b] + ddg[m][b][l][a] - ddg[m][l][a][b]);
      }
  double G2[3][3][3];
  for (int kk = 0; kk < 3; kk++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double s = 0.0;
        for (int l = 0; l < 3; l++) s += gu[kk][l] * G1[l][a][b];
        G2[kk][a][b] = s;
      }
  /* d_m gamma^kl */
  double dgu[3][3][3];
  for (int m = 0; m < 3; m++)
    for (int kk = 0; kk < 3; kk++)
      for (int l = 0; l < 3; l++) {
        double s = 0.0;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) s -= gu[kk][a] * gu[l][b] * dg[m][a][b];
        dgu[m][kk][l] = s;
      }
  /* d_m Gamma^k_ij = d_m gamma^kl Gamma_lij + gamma^kl d_m Gamma_lij */
  double dG2[3][3][3][3];
  for (int m = 0; m < 3; m++)
    for (int kk = 0; kk < 3; kk++)
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          double s = 0.0;
          for (int l = 0; l < 3; l++) s += dgu[m][kk][l] * G1[l][a][b] + gu[kk][l] * dG1[m][l][a][b];
          dG2[m][kk][a][b] = s;
        }
  double R = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0;
      for (int kk = 0; kk < 3; kk++) s += dG2[kk][kk][a][b] - dG2[b][kk][a][kk];
      for (int kk = 0; kk < 3; kk++)
        for (int l = 0; l < 3; l++) s += G2[kk][kk][l] * G2[l][a][b] - G2[kk][b][l] * G2[l][a][kk];
      R += gu[a][b] * s;
    }
  double Kud[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0;
      for (int l = 0; l < 3; l++) s += gu[a][l] * K[l][b];
      Kud[a][b] = s;
    }
  double trK = 0.0, KK = 0.0;
  for (int a = 0; a < 3; a++) trK += Kud[a][a];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) KK += Kud[a][b] * Kud[b][a];
  out[0] = R - KK + trK * trK;
  /* nabla_m K_ab = d_m K_ab - Gamma^l_ma K_lb - Gamma^l_mb K_al */
  double DK[3][3][3];
  for (int m = 0; m < 3; m++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double s = dKd[m][a][b];
        for (int l = 0; l < 3; l++) s -= G2[l][m][a] * K[l][b] + G2[l][m][b] * K[a][l];
        DK[m][a][b] = s;
      }
  for (int a = 0; a < 3; a++) {
    double s = 0.0;
    for (int jj = 0; jj < 3; jj++)
      for (int kk = 0; kk < 3; kk++) s += gu[jj][kk] * (DK[kk][a][jj] - DK[a][jj][kk]);
    out[1 + a] = s;
  }
}

/* Matter terms of the constraints (Sec. "Other analysis modules" with the
 * normalisation of the ADM mass integrand): H gets -16 pi E, M_i gets
 * -8 pi S_i, with alpha and beta^i of the state at the point. */
static void constraint_sources(const ocfg* c, const double* st, size_t id, double o[4]) {
  if (!c->tmunu) return;
  const size_t S = npts(c);
  double alpha = st[(size_t)F_ALP * S + id], beta[3], gdummy[3][3] = {{0.0}}, E, Si[3], Sij[3][3], Sm;
  for (int a = 0; a < 3; a++) beta[a] = st[(size_t)(F_BETA + a) * S + id];
  matter_projections(c, id, alpha, beta, gdummy, &E, Si, Sij, &Sm);
  o[0] -= 16.0 * M_PI * E;
  for (int a = 0; a < 3; a++) o[1 + a] -= 8.0 * M_PI * Si[a];
}

/* Constraint norms over interior points.  out16: L2 H, Mx, My, Mz, Linf H,
 * Mx, My, Mz over all interior points, then the same over points farther
 * than r_excise from every puncture.  L2 is the root mean square.  Hgrid and
 * Mgrid (may be NULL) receive the pointwise values (Mgrid: 3 components). */
int oracle_constraints(const ocfg* c, const double* st, double* out16, double* Hgrid,
                       double* Mgrid) {
  const size_t S = npts(c);
  double* gam6 = (double*)malloc(6 * S * sizeof(double));
  double* K6 = (double*)malloc(6 * S * sizeof(double));
  if (!gam6 || !K6) {
    free(gam6); free(K6);
    return 2;
  }
  adm_grids(c, st, gam6, K6);
  double sum[2][4] = {{0}}, mx[2][4] = {{0}};
  long cnt[2] = {0, 0};
  for (int k = GH; k < GH + c->n[2]; k++)
    for (int j = GH; j < GH + c->n[1]; j++)
      for (int i = GH; i < GH + c->n[0]; i++) {
        double o[4];
        constraints_point(c, gam6, K6, i, j, k, o);
        size_t id = pidx(c, i, j, k);
        constraint_sources(c, st, id, o);
        if (Hgrid) Hgrid[id] = o[0];
        if (Mgrid)
          for (int a = 0; a < 3; a++) Mgrid[(size_t)a * S + id] = o[1 + a];
        double x = coord(c, 0, i), y = coord(c, 1, j), z = coord(c, 2, k);
        int outside = 1;
        for (int a = 0; a < c->npunct; a++) {
          double dx = x - c->punct[a][1], dy = y - c->punct[a][2], dz = z - c->punct[a][3];
          if (sqrt(dx * dx + dy * dy + dz * dz) <= c->r_excise) outside = 0;
        }
        for (int set = 0; set < 2; set++) {
          if (set == 1 && !outside) continue;
          cnt[set]++;
          for (int q = 0; q < 4; q++) {
            sum[set][q] += o[q] * o[q];
            if (fabs(o[q]) > mx[set][q]) mx[set][q] = fabs(o[q]);
          }
        }
      }
  for (int set = 0; set < 2; set++)
    for (int q = 0; q < 4; q++) {
      out16[set * 8 + q] = cnt[set] ? sqrt(sum[set][q] / (double)cnt[set]) : 0.0;
      out16[set * 8 + 4 + q] = mx[set][q];
    }
  free(gam6);
  free(K6);
  return 0;
}

/* Constraints at a list of interior points (o[p*4 + q]). */
int oracle_constraints_points(const ocfg* c, const double* st, int np, const int* ijk,
                              double* out) {
  const size_t S = npts(c);
  double* gam6 = (double*)malloc(6 * S * sizeof(double));
  double* K6 = (double*)malloc(6 * S * sizeof(double));
  if (!gam6 || !K6) {
    free(gam6); free(K6);
    return 2;
  }
  adm_grids(c, st, gam6, K6);
  for (int p = 0; p < np; p++)
  {
    constraints_point(c, gam6, K6, ijk[3 * p], ijk[3 * p + 1], ijk[3 * p + 2], out + 4 * p);
    constraint_sources(c, st, pidx(c, ijk[3 * p], ijk[3 * p + 1], ijk[3 * p + 2]), out + 4 * p);
  }
  free(gam6);
  free(K6);
  return 0;
}

/* ------------------------------------------ ADM mass and angular momentum
 * Sec. "Masses and Momenta" (volume-integral form of ML_ADMQuantities):
 *   M   = 1/(16 pi) int d^3x [ e^{5 phi}(16 pi E + At_ij At^ij - (2/3) K^2)
 *                              - e^{phi} Rt ]
 *   J_i = 1/(8 pi) eps_ij^k int d^3x e^{6 phi} [ At^j_k + (2/3) x^j Dt_k K
 *                              - (1/2) x^j At_ln d_k gt^{ln} + 8 pi x^j S_k ]
 * with E and S_k the matter projections when T_{mu nu} is given (else 0).
 * Readings:
 *  - Rt = gt^ij Rt_ij with the same Rt_ij as the right-hand side (the
 *    evolved Gt^k in gt_k(i d_j) Gt^k, the metric-derived d_l gt^{lk}
 *    elsewhere), from the same 4th-order stencils;
 *  - Dt_k K = d_k K (a scalar), 4th-order centred;
 *  - d_k gt^{ln} = -gt^{la} gt^{nb} d_k gt_ab (derivative of the inverse);
 *  - At^j_k = gt^{jl} At_lk, At^ij = gt^ia gt^jb At_ab;
 *  - eps_ij^k is the Levi-Civita symbol of the Cartesian grid coordinates,
 *    and x^j the grid coordinates themselves (origin at x = 0);
 *  - e^{phi} = W^{-1/2} in the W variant, with W floored at w_floor there
 *    (the only place it divides);
 *  - the integral is the midpoint sum h^3 sum over the interior points (each
 *    point is the centre of a cell of the interior block), over all of them
 *    and over the points farther than r_excise from every puncture.
 * Pins: for exact vacuum data the integrands are divergences (the
 * Hamiltonian and momentum constraints), -(1/2 pi) d_i(gt^ij d_j psi) and
 * (1/8 pi) eps_ijk d_l(x^j psi^6 At^l_k) with psi = e^{phi}, which the tests
 * evaluate exactly and compare at 4th order; the box sums converge to the
 * corresponding surface integrals.
 */
static void adm_density_point(const ocfg* c, const double* st, int i, int j, int k,
                              double out[4]) {
  const size_t S = npts(c);
  const size_t id = pidx(c, i, j, k);
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  const double h = c->h;
  const double* P0 = st + id;
  double chi = P0[(size_t)F_CHI * S];
  double trK = P0[(size_t)F_TRK * S];
  double g[3][3], A[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      g[a][b] = P0[(size_t)(F_GT + SYM[a][b]) * S];
      A[a][b] = P0[(size_t)(F_AT + SYM[a][b]) * S];
    }
  double dg[3][3][3], ddg[3][3][3][3], dGt[3][3], dK[3];
  for (int kk = 0; kk < 3; kk++) {
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        const double* p = P0 + (size_t)(F_GT + SYM[a][b]) * S;
        dg[kk][a][b] = st_d1(p, str[kk], h);
        for (int l = 0; l < 3; l++) ddg[kk][l][a][b] = st_dd(p, str, kk, l, h);
      }
    for (int a = 0; a < 3; a++) dGt[kk][a] = st_d1(P0 + (size_t)(F_GAM + a) * S, str[kk], h);
    dK[kk] = st_d1(P0 + (size_t)F_TRK * S, str[kk], h);
  }
  double gu[3][3];
  inv3(g, gu);
  double G1[3][3][3], G2[3][3][3], dgu[3];
  for (int kk = 0; kk < 3; kk++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++)
        G1[kk][a][b] = 0.5 * (dg[a][kk][b] + dg[b][kk][a] - dg[kk][a][b]);
  for (int kk = 0; kk < 3; kk++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double s = 0.0;
        for (int l = 0; l < 3; l++) s += gu[kk][l] * G1[l][a][b];
        G2[kk][a][b] = s;
      }
  for (int kk = 0; kk < 3; kk++) {
    double s = 0.0;
    for (int l = 0; l < 3; l++)
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) s -= gu[l][a] * gu[kk][b] * dg[l][a][b];
    dgu[kk] = s;
  }
  /* Rt_ij exactly as in the right-hand side, then its trace */
  double Rt_trace = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0;
      for (int kk = 0; kk < 3; kk++)
        for (int l = 0; l < 3; l++) s += -0.5 * gu[kk][l] * ddg[kk][l][a][b];
      for (int kk = 0; kk < 3; kk++)
        s += 0.5 * (g[kk][a] * dGt[b][kk] + g[kk][b] * dGt[a][kk]);
      for (int kk = 0; kk < 3; kk++)
        s -= 0.5 * (G1[a][b][kk] + G1[b][a][kk]) * dgu[kk];
      for (int l = 0; l < 3; l++)
        for (int m = 0; m < 3; m++) {
          double t = 0.0;
          for (int kk = 0; kk < 3; kk++)
            t += G2[kk][l][a] * G1[b][kk][m] + G2[kk][l][b] * G1[a][kk][m] +
                 G2[kk][a][m] * G1[kk][l][b];
          s += gu[l][m] * t;
        }
      Rt_trace += gu[a][b] * s;
    }
  /* e^{phi} */
  double ephi;
  if (c->use_w) {
    double Wd = chi > c->w_floor ? chi : c->w_floor;
    ephi = 1.0 / sqrt(Wd);
  } else {
    ephi = exp(chi);
  }
  double e5 = pow(ephi, 5.0), e6 = pow(ephi, 6.0);
  /* At^ij, At^j_k, At_ij At^ij */
  double Au[3][3], Am[3][3], AA = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0, m = 0.0;
      for (int p = 0; p < 3; p++) {
        m += gu[a][p] * A[p][b];
        for (int q = 0; q < 3; q++) s += gu[a][p] * gu[b][q] * A[p][q];
      }
      Au[a][b] = s;
      Am[a][b] = m;
    }
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) AA += A[a][b] * Au[a][b];
  /* matter: E and S_k (zero in vacuum) */
  double Em = 0.0, Sk[3] = {0.0, 0.0, 0.0};
  if (c->tmunu) {
    double alpha = P0[(size_t)F_ALP * S], beta[3], gdummy[3][3] = {{0.0}}, Sij[3][3], Sm;
    for (int a = 0; a < 3; a++) beta[a] = P0[(size_t)(F_BETA + a) * S];
    matter_projections(c, id, alpha, beta, gdummy, &Em, Sk, Sij, &Sm);
  }
  out[0] = (e5 * (16.0 * M_PI * Em + AA - (2.0 / 3.0) * trK * trK) - ephi * Rt_trace) / (16.0 * M_PI);
  /* d_k gt^{ln} and At_ln d_k gt^{ln} */
  double AdG[3];
  for (int kk = 0; kk < 3; kk++) {
    double s = 0.0;
    for (int l = 0; l < 3; l++)
      for (int n = 0; n < 3; n++) {
        double dgtu = 0.0;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) dgtu -= gu[l][a] * gu[n][b] * dg[kk][a][b];
        s += A[l][n] * dgtu;
      }
    AdG[kk] = s;
  }
  const double x[3] = {coord(c, 0, i), coord(c, 1, j), coord(c, 2, k)};
  for (int ii = 0; ii < 3; ii++) {
    double s = 0.0;
    for (int jj = 0; jj < 3; jj++)
      for (int kk = 0; kk < 3; kk++) {
        /* Levi-Civita symbol eps_{ii jj kk} */
        double eps = (double)((ii - jj) * (jj - kk) * (kk - ii)) / 2.0;
        if (eps == 0.0) continue;
        double v = Am[jj][kk] + (2.0 / 3.0) * x[jj] * dK[kk] - 0.5 * x[jj] * AdG[kk] +
                   8.0 * M_PI * x[jj] * Sk[kk];
        s += eps * e6 * v;
      }
    out[1 + ii] = s / (8.0 * M_PI);
  }
}

/* Volume integrals M, J_x, J_y, J_z over all interior points (out8[0..3])
 * and over the points farther than r_excise from every puncture
 * (out8[4..7]).  dens (may be NULL) receives the four integrands at every
 * interior point, (4, stored points); other points are left untouched. */
int oracle_adm_integrals(const ocfg* c, const double* st, double* out8, double* dens) {
  const size_t S = npts(c);
  double sum[2][4] = {{0}};
  for (int k = GH; k < GH + c->n[2]; k++)
    for (int j = GH; j < GH + c->n[1]; j++)
      for (int i = GH; i < GH + c->n[0]; i++) {
        double o[4];
        adm_density_point(c, st, i, j, k, o);
        size_t id = pidx(c, i, j, k);
        if (dens)
          for (int q = 0; q < 4; q++) dens[(size_t)q * S + id] = o[q];
        double x = coord(c, 0, i), y = coord(c, 1, j), z = coord(c, 2, k);
        int outside = 1;
        for (int a = 0; a < c->npunct; a++) {
          double dx = x - c->punct[a][1], dy = y - c->punct[a][2], dz = z - c->punct[a][3];
          if (sqrt(dx * dx + dy * dy + dz * dz) <= c->r_excise) outside = 0;
        }
        for (int q = 0; q < 4; q++) {
          sum[0][q] += o[q];
          if (outside) sum[1][q] += o[q];
        }
      }
  const double vol = c->h * c->h * c->h;
  for (int set = 0; set < 2; set++)
    for (int q = 0; q < 4; q++) out8[set * 4 + q] = sum[set][q] * vol;
  return 0;
}

/* ------------------------------------------------------ puncture tracking
 * Sec. "Object tracking": each puncture moves by dx^i/dt = -beta^i at its
 * position, integrated by forward Euler, x_{n+1} = x_n - dt beta^i(t_n, x_n),
 * with the shift of the state at the start of the step.  Readings: the
 * shift is interpolated by the tensor product of 4-point Lagrange
 * polynomials (cubic in each direction) on the stored points i0-1 .. i0+2,
 * i0 the stored point at or below the position; the stencil is shifted to
 * stay inside the stored block (then the polynomial extrapolates).
 */
static double lagrange4(int m, double u) {
  /* basis polynomial of node m in {-1, 0, 1, 2}, evaluated at u */
  double v = 1.0;
  for (int n = -1; n <= 2; n++)
    if (n != m) v *= (u - n) / (double)(m - n);
  return v;
}

static void interp_setup(const ocfg* c, int d, double x, int* i0, double* u) {
  double s = (x - coord(c, d, 0)) / c->h;  /* position in stored-index units */
  int b = (int)floor(s);
  if (b < 1) b = 1;
  if (b > dimx(c, d) - 3) b = dimx(c, d) - 3;
  *i0 = b;
  *u = s - b;
}

/* Tricubic Lagrange interpolation of grid function f at (x, y, z). */
double oracle_interp(const ocfg* c, const double* f, const double xyz[3]) {
  int i0[3];
  double u[3];
  for (int d = 0; d < 3; d++) interp_setup(c, d, xyz[d], &i0[d], &u[d]);
  double s = 0.0;
  for (int mk = -1; mk <= 2; mk++)
    for (int mj = -1; mj <= 2; mj++)
      for (int mi = -1; mi <= 2; mi++)
        s += lagrange4(mi, u[0]) * lagrange4(mj, u[1]) * lagrange4(mk, u[2]) *
             f[pidx(c, i0[0] + mi, i0[1] + mj, i0[2] + mk)];
  return s;
}

/* One Euler step of every puncture: pos[a] = {m, x, y, z}, a < np, updated in
 * place from the shift of st. */
void oracle_track_step(const ocfg* c, const double* st, int np, double* pos, double dt) {
  const size_t S = npts(c);
  for (int a = 0; a < np; a++) {
    double* p = pos + 4 * a;
    double xyz[3] = {p[1], p[2], p[3]};
    double beta[3];
    for (int d = 0; d < 3; d++) beta[d] = oracle_interp(c, st + (size_t)(F_BETA + d) * S, xyz);
    for (int d = 0; d < 3; d++) p[1 + d] = xyz[d] - dt * beta[d];
  }
}

/* ------------------------------------------------------------ Weyl scalar
 * Sec. "Gravitational Waves" (WeylScal4): Psi4 = C_abcd n^a mb^b n^c mb^d for
 * the fiducial tetrad l = (u + r)/sqrt2, n = (u - r)/sqrt2,
 * m = (theta + i phi)/sqrt2, u the unit normal of the slice, from the
 * projections of the curvature onto the slice.  Readings:
 *  - index 0 of the printed formula is the component along u, so n^0 = 1/sqrt2,
 *    the spatial part of n is -r/sqrt2, and mb^0 = 0 (the triad is spatial),
 *    which removes every term with mb^0;
 *  - the three projections (vacuum, K_ij = -grad_i u_j):
 *      R_ijkl = 3R_ijkl + K_ik K_jl - K_il K_jk                (Gauss)
 *      R_0jkl = D_k K_jl - D_l K_jk                            (Codazzi)
 *      R_0j0l = 3R_jl + K K_jl - K_jm K^m_l                    (Ricci, vacuum)
 *    with 3R_ijkl = 1/2 (d_j d_k g_il + d_i d_l g_jk - d_i d_k g_jl
 *    - d_j d_l g_ik) + g_mn (G^m_jk G^n_il - G^m_jl G^n_ik) and 3R_jl =
 *    g^ik 3R_ijkl, all from 4th-order stencils of the ADM fields formed
 *    pointwise (as for the constraints);
 *  - the triad starts from r = x^i, phi = (-y, x, 0),
 *    theta^i = sqrt(det g) g^ik eps_klm phi^l r^m (x^i the grid coordinates,
 *    origin at 0), and is made orthonormal in g_ij by Gram-Schmidt in the
 *    order phi, r, theta;
 *  - on the z axis (phi = 0) the triad is undefined: Psi4 = 0 there.
 * Pin: the exact 4-Riemann tensor of exact spacetimes (Taylor jets of the
 * 4-metric) contracted with the same tetrad, at 4th order; flat space in
 * curved slicings gives 0; the triad is the spherical one for a flat metric.
 */
static void psi4_point(const ocfg* c, const double* gam6, const double* K6, int i, int j, int k,
                       double out[2]) {
  const size_t S = npts(c);
  const size_t id = pidx(c, i, j, k);
  const ptrdiff_t str[3] = {1, dimx(c, 0), (ptrdiff_t)dimx(c, 0) * dimx(c, 1)};
  const double h = c->h;
  double g[3][3], K[3][3], dg[3][3][3], ddg[3][3][3][3], dK[3][3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      const double* pg = gam6 + (size_t)SYM[a][b] * S + id;
      const double* pk = K6 + (size_t)SYM[a][b] * S + id;
      g[a][b] = pg[0];
      K[a][b] = pk[0];
      for (int m = 0; m < 3; m++) {
        dg[m][a][b] = st_d1(pg, str[m], h);
        dK[m][a][b] = st_d1(pk, str[m], h);
        for (int n = 0; n < 3; n++) ddg[m][n][a][b] = st_dd(pg, str, m, n, h);
      }
    }
  double gu[3][3];
  inv3(g, gu);
  /* Christoffel symbols G^m_ij */
  double G[3][3][3];
  for (int m = 0; m < 3; m++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double s = 0.0;
        for (int l = 0; l < 3; l++) s += 0.5 * gu[m][l] * (dg[a][l][b] + dg[b][a][l] - dg[l][a][b]);
        G[m][a][b] = s;
      }
  /* 3-Riemann R_ijkl (all indices down) */
  double R4[3][3][3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int cc = 0; cc < 3; cc++)
        for (int d = 0; d < 3; d++) {
          double s = 0.5 * (ddg[b][cc][a][d] + ddg[a][d][b][cc] - ddg[a][cc][b][d] - ddg[b][d][a][cc]);
          for (int m = 0; m < 3; m++)
            for (int n = 0; n < 3; n++) s += g[m][n] * (G[m][b][cc] * G[n][a][d] - G[m][b][d] * G[n][a][cc]);
          R4[a][b][cc][d] = s;
        }
  double Ric[3][3];
  for (int b = 0; b < 3; b++)
    for (int d = 0; d < 3; d++) {
      double s = 0.0;
      for (int a = 0; a < 3; a++)
        for (int cc = 0; cc < 3; cc++) s += gu[a][cc] * R4[a][b][cc][d];
      Ric[b][d] = s;
    }
  double trK = 0.0, Kud[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      trK += gu[a][b] * K[a][b];
      double s = 0.0;
      for (int m = 0; m < 3; m++) s += gu[a][m] * K[m][b];
      Kud[a][b] = s; /* K^a_b */
    }
  /* D_k K_jl */
  double DK[3][3][3];
  for (int m = 0; m < 3; m++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double s = dK[m][a][b];
        for (int l = 0; l < 3; l++) s -= G[l][m][a] * K[l][b] + G[l][m][b] * K[a][l];
        DK[m][a][b] = s;
      }
  /* projections */
  double Rs[3][3][3][3], R0[3][3][3], R00[3][3];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int cc = 0; cc < 3; cc++)
        for (int d = 0; d < 3; d++)
          Rs[a][b][cc][d] = R4[a][b][cc][d] + K[a][cc] * K[b][d] - K[a][d] * K[b][cc];
  for (int b = 0; b < 3; b++)
    for (int cc = 0; cc < 3; cc++)
      for (int d = 0; d < 3; d++) R0[b][cc][d] = DK[cc][b][d] - DK[d][b][cc];
  for (int b = 0; b < 3; b++)
    for (int d = 0; d < 3; d++) {
      double s = Ric[b][d] + trK * K[b][d];
      for (int m = 0; m < 3; m++) s -= K[b][m] * Kud[m][d];
      R00[b][d] = s;
    }
  /* fiducial triad */
  const double x[3] = {coord(c, 0, i), coord(c, 1, j), coord(c, 2, k)};
  double rv[3] = {x[0], x[1], x[2]};
  double pv[3] = {-x[1], x[0], 0.0};
  double tv[3];
  const double sdet = sqrt(det3(g));
  for (int a = 0; a < 3; a++) {
    double s = 0.0;
    for (int kk = 0; kk < 3; kk++)
      for (int l = 0; l < 3; l++)
        for (int m = 0; m < 3; m++) {
          double eps = (double)((kk - l) * (l - m) * (m - kk)) / 2.0;
          s += sdet * gu[a][kk] * eps * pv[l] * rv[m];
        }
    tv[a] = s;
  }
#define DOT(u, v) (g[0][0] * u[0] * v[0] + g[0][1] * u[0] * v[1] + g[0][2] * u[0] * v[2] + \
                   g[1][0] * u[1] * v[0] + g[1][1] * u[1] * v[1] + g[1][2] * u[1] * v[2] + \
                   g[2][0] * u[2] * v[0] + g[2][1] * u[2] * v[1] + g[2][2] * u[2] * v[2])
  double pp = DOT(pv, pv);
  if (!(pp > 0.0)) {
    out[0] = out[1] = 0.0;
    return;
  }
  for (int a = 0; a < 3; a++) pv[a] /= sqrt(pp);
  double rp = DOT(rv, pv);
  for (int a = 0; a < 3; a++) rv[a] -= rp * pv[a];
  double rr = DOT(rv, rv);
  for (int a = 0; a < 3; a++) rv[a] /= sqrt(rr);
  double tp = DOT(tv, pv), tr = DOT(tv, rv);
  for (int a = 0; a < 3; a++) tv[a] -= tp * pv[a] + tr * rv[a];
  double tt = DOT(tv, tv);
  for (int a = 0; a < 3; a++) tv[a] /= sqrt(tt);
#undef DOT
  /* tetrad components: n^0 = 1/sqrt2, n^i = -r^i/sqrt2, mb^i = (theta^i - i phi^i)/sqrt2 */
  const double s2 = 1.0 / sqrt(2.0);
  double complex mb[3];
  double n[3];
  for (int a = 0; a < 3; a++) {
    n[a] = -s2 * rv[a];
    mb[a] = s2 * (tv[a] - _Complex_I * pv[a]);
  }
  const double n0 = s2;
  double complex psi = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int cc = 0; cc < 3; cc++)
        for (int d = 0; d < 3; d++) psi += Rs[a][b][cc][d] * n[a] * mb[b] * n[cc] * mb[d];
  for (int b = 0; b < 3; b++)
    for (int cc = 0; cc < 3; cc++)
      for (int d = 0; d < 3; d++) psi += 2.0 * R0[b][cc][d] * n0 * mb[b] * n[cc] * mb[d];
  for (int b = 0; b < 3; b++)
    for (int d = 0; d < 3; d++) psi += R00[b][d] * n0 * mb[b] * n0 * mb[d];
  out[0] = creal(psi);
  out[1] = cimag(psi);
}

/* Psi4 at every interior point: out2 (2, stored points) real and imaginary
 * parts; other points are left untouched.  Returns 2 on allocation failure. */
int oracle_psi4(const ocfg* c, const double* st, double* out2) {
  const size_t S = npts(c);
  double* gam6 = (double*)malloc(6 * S * sizeof(double));
  double* K6 = (double*)malloc(6 * S * sizeof(double));
  if (!gam6 || !K6) {
    free(gam6); free(K6);
    return 2;
  }
  adm_grids(c, st, gam6, K6);
  for (int k = GH; k < GH + c->n[2]; k++)
    for (int j = GH; j < GH + c->n[1]; j++)
      for (int i = GH; i < GH + c->n[0]; i++) {
        double o[2];
        psi4_point(c, gam6, K6, i, j, k, o);
        size_t id = pidx(c, i, j, k);
        out2[id] = o[0];
        out2[S + id] = o[1];
      }
  free(gam6);
  free(K6);
  return 0;
}
