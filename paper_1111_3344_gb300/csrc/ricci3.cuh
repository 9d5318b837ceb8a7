// Christoffel symbols and Ricci tensor of a 3-metric g_ij from its first and
// second differences, float64, for the analysis kernels (constraints and Psi4:
// Ricci tensor of gamma_ij; ADM integrals: Christoffel symbols of gt_ij;
// arXiv:1111.3344, Sec. "Other analysis modules", Sec. "Masses and Momenta",
// Sec. "Gravitational Waves").
//
//   Gamma_kij   = (d_i g_kj + d_j g_ki - d_k g_ij) / 2,   Gamma^k_ij = g^ks Gamma_sij
//   R_ij = 1/2 g^kl (d_k d_j g_il + d_i d_l g_kj - d_k d_l g_ij - d_i d_j g_kl)
//          + g^kl (Gamma^m_il Gamma_mkj - Gamma^m_ij Gamma_mkl)
//
// The sums are arranged with exact identities to cut float64 work (about 350
// operations for R_ij instead of about 600 term by term):
//  - the terms of Gamma_kij that cancel when two indices coincide are left out;
//  - g^kl d_k d_l g_ij and g^kl d_i d_j g_kl are contractions over the six
//    symmetric pairs (off-diagonal weights doubled);
//  - the two mixed second-difference terms are V_ij + V_ji with
//    V_ij = g^kl d_k d_j g_il;
//  - g^kl Gamma^m_il Gamma_mkj = Gamma^m_il H_m^l_j with H_m^l_j = g^lk Gamma_mkj,
//    and g^kl Gamma^m_ij Gamma_mkl = Gamma^m_ij Gamma_m with Gamma_m = g^kl Gamma_mkl.
// Indices: dg[d][m] = d_d g_m and ddg[pq][m] = d_p d_q g_m, symmetric pairs
// m, pq stored as 6 components (sym()).
#pragma once
#include "bssn_internal.cuh"

namespace bssn {

__device__ __forceinline__ void christoffel3(const double gu[6], const double dg[3][6], double G1[3][6],
                                             double G2[3][6]) {
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++) {
        double v;
        if (a == b && k == a)
          v = 0.5 * dg[a][sym(a, a)];
        else if (a == b)
          v = fma(-0.5, dg[k][sym(a, a)], dg[a][sym(k, a)]);
        else if (k == a)
          v = 0.5 * dg[b][sym(a, a)];
        else if (k == b)
          v = 0.5 * dg[a][sym(b, b)];
        else
          v = 0.5 * (dg[a][sym(k, b)] + dg[b][sym(k, a)] - dg[k][sym(a, b)]);
        G1[k][sym(a, b)] = v;
      }
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int m = 0; m < 6; m++)
      G2[k][m] = gu[sym(k, 0)] * G1[0][m] + gu[sym(k, 1)] * G1[1][m] + gu[sym(k, 2)] * G1[2][m];
}

__device__ __forceinline__ void ricci3(const double gu[6], const double ddg[6][6], const double G1[3][6],
                                       const double G2[3][6], double Ric[6]) {
  double g2u[6];  // g^kl with the off-diagonal entries doubled
#pragma unroll
  for (int m = 0; m < 6; m++) g2u[m] = (m == 0 || m == 3 || m == 5) ? gu[m] : 2.0 * gu[m];
  // a_ij = g^kl d_k d_l g_ij, b_ij = g^kl d_i d_j g_kl
  double a[6], b[6];
#pragma unroll
  for (int m = 0; m < 6; m++) {
    double sa = 0.0, sb = 0.0;
#pragma unroll
    for (int q = 0; q < 6; q++) {
      sa = fma(g2u[q], ddg[q][m], sa);
      sb = fma(g2u[q], ddg[m][q], sb);
    }
    a[m] = sa;
    b[m] = sb;
  }
  // V_ij = g^kl d_k d_j g_il
  double V[3][3];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 3; k++)
#pragma unroll
        for (int l = 0; l < 3; l++) s = fma(gu[sym(k, l)], ddg[sym(k, j)][sym(i, l)], s);
      V[i][j] = s;
    }
  // H[m][l][j] = g^lk Gamma_mkj, Gl[m] = g^kl Gamma_mkl
  double H[3][3][3], Gl[3];
#pragma unroll
  for (int m = 0; m < 3; m++) {
#pragma unroll
    for (int l = 0; l < 3; l++)
#pragma unroll
      for (int j = 0; j < 3; j++)
        H[m][l][j] = gu[sym(l, 0)] * G1[m][sym(0, j)] + gu[sym(l, 1)] * G1[m][sym(1, j)] +
                     gu[sym(l, 2)] * G1[m][sym(2, j)];
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 6; q++) s = fma(g2u[q], G1[m][q], s);
    Gl[m] = s;
  }
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = i; j < 3; j++) {
      const int ij = sym(i, j);
      double s = 0.5 * ((V[i][j] + V[j][i]) - (a[ij] + b[ij]));
#pragma unroll
      for (int m = 0; m < 3; m++) {
#pragma unroll
        for (int l = 0; l < 3; l++) s = fma(G2[m][sym(i, l)], H[m][l][j], s);
        s = fma(-G2[m][ij], Gl[m], s);
      }
      Ric[ij] = s;
    }
}

}  // namespace bssn
