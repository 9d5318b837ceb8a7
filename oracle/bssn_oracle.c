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
 * convergence, the outgoing-wave Sommerfeld condition with its power-law
 * correction (an exact C/r^2 tail carried outwards), X0 per variable (flat
 * space stays exactly flat) and v0 = sqrt(2) for alpha and K (the speed at
 * which 1+log slicing carries a lapse pulse).  v0 = 1 for the other fields and
 * the initial lapse are readings of an under-specified passage: parity of
 * those two choices is unpinned.
 */
#include <complex.h>
#undef I /* the imaginary unit is written _Complex_I below */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* Arithmetic type of the shared right-hand-side header: plain float64. */
typedef double real;
#include "bssn_rhs.h"

size_t oracle_npoints(const ocfg* c) { return npts(c); }

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
