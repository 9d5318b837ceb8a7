// Weyl scalar Psi4 (arXiv:1111.3344, Sec. "Gravitational Waves", WeylScal4):
// Psi4 = C_abcd n^a mb^b n^c mb^d for the fiducial tetrad n = (u - r)/sqrt2,
// mb = (theta - i phi)/sqrt2, from the projections of the vacuum curvature
// onto the slice (index 0 = along the unit normal u, so n^0 = 1/sqrt2 and
// mb^0 = 0):
//   R_ijkl n mb n mb + 2 n^0 R_0jkl mb n mb + (n^0)^2 R_0j0l mb mb
//   R_ijkl = 3R_ijkl + K_ik K_jl - K_il K_jk,  R_0jkl = D_k K_jl - D_l K_jk,
//   R_0j0l = 3R_jl + K K_jl - K_jm K^m_l.
// The triad starts from r = x^i, phi = (-y, x, 0),
// theta^i = sqrt(det g) g^ik eps_klm phi^l r^m and is made orthonormal in g_ij
// by Gram-Schmidt in the order phi, r, theta; Psi4 = 0 where phi = 0.
//
// Formulation: in three dimensions the Riemann tensor is fixed by the Ricci
// tensor, 3R_ijkl = g_ik R_jl + g_jl R_ik - g_il R_jk - g_jk R_il
// - (R/2)(g_ik g_jl - g_il g_jk), and for the orthonormal triad n.n = 1/2,
// mb.mb = n.mb = 0, so 3R(n, mb, n, mb) = R(mb, mb)/2 and
//   Psi4 = R(mb,mb) + K(n,n) K(mb,mb) - K(n,mb)^2
//          + sqrt2 [ n^k D_k K(mb,mb) - mb^l D_l K(mb,n) ]
//          + (K K(mb,mb) - (K.K)(mb,mb)) / 2,
// evaluated with the triad's real vectors (mb = (t - i p)/sqrt2, n = -r/sqrt2)
// so that only the Ricci tensor (6 components) is formed.  The ADM fields
// gamma_ij = e^{4 phi} gt_ij, K_ij = e^{4 phi}(At_ij + gt_ij K/3) are formed at
// every stencil point and differenced with the 4th-order stencils.  Float64
// in every precision mode; one thread per interior point.
#include "bssn_internal.cuh"
#include "ricci3.cuh"

namespace bssn {

namespace {

constexpr int PB = 128;  // threads per block

template <bool PRE>
__device__ __forceinline__ void adm_fields(const Grid& g, const double* __restrict__ y,
                                           const double* __restrict__ adm, long long id, double gam[6],
                                           double K[6], bool needK) {
  const long long fs = g.fstride;
  if constexpr (PRE) {  // precomputed by launch_adm_fields with the operations below
#pragma unroll
    for (int m = 0; m < 6; m++) {
      gam[m] = __ldg(adm + m * fs + id);
      if (needK) K[m] = __ldg(adm + (6 + m) * fs + id);
    }
    return;
  }
  const double chi = __ldg(y + F_CHI * fs + id);
  const double e4 = g.use_w ? 1.0 / (chi * chi) : exp(4.0 * chi);
  const double tr3 = needK ? __ldg(y + F_TRK * fs + id) * (1.0 / 3.0) : 0.0;
#pragma unroll
  for (int m = 0; m < 6; m++) {
    const double gt = __ldg(y + (F_GT + m) * fs + id);
    gam[m] = e4 * gt;
    if (needK) K[m] = e4 * (__ldg(y + (F_AT + m) * fs + id) + gt * tr3);
  }
}

// bilinear form of a symmetric 6-component tensor
__device__ __forceinline__ double bil(const double T[6], const double a[3], const double b[3]) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) s = fma(T[sym(i, j)] * a[i], b[j], s);
  return s;
}

template <bool PRE>
__device__ void psi4_point(const Grid& g, const double* __restrict__ y, const double* __restrict__ adm,
                           long long id, const double x[3], double out[2]) {
  const long long sd[3] = {1, g.pitch, g.plane};
  const double i12h = g.i12h, i12h2 = g.i12h2, i144h2 = g.i144h2;
  double g0[6], k0[6];
  adm_fields<PRE>(g, y, adm, id, g0, k0, true);
  double dg[3][6], dk[3][6], ddg[6][6];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double gp1[6], gm1[6], gp2[6], gm2[6], kp1[6], km1[6], kp2[6], km2[6];
    adm_fields<PRE>(g, y, adm, id + sd[d], gp1, kp1, true);
    adm_fields<PRE>(g, y, adm, id - sd[d], gm1, km1, true);
    adm_fields<PRE>(g, y, adm, id + 2 * sd[d], gp2, kp2, true);
    adm_fields<PRE>(g, y, adm, id - 2 * sd[d], gm2, km2, true);
#pragma unroll
    for (int m = 0; m < 6; m++) {
      dg[d][m] = fma(8.0, gp1[m] - gm1[m], -(gp2[m] - gm2[m])) * i12h;
      dk[d][m] = fma(8.0, kp1[m] - km1[m], -(kp2[m] - km2[m])) * i12h;
      ddg[sym(d, d)][m] = fma(-30.0, g0[m], fma(16.0, gp1[m] + gm1[m], -(gp2[m] + gm2[m]))) * i12h2;
    }
  }
  {
    const double c[4] = {1.0, -8.0, 8.0, -1.0};
    const int off[4] = {-2, -1, 1, 2};
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a + 1; b < 3; b++) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        double dummy[6];
#pragma unroll
        for (int p = 0; p < 4; p++)
#pragma unroll
          for (int q = 0; q < 4; q++) {
            double gv[6];
            adm_fields<PRE>(g, y, adm, id + off[p] * sd[a] + off[q] * sd[b], gv, dummy, false);
            const double w = c[p] * c[q];
#pragma unroll
            for (int m = 0; m < 6; m++) acc[m] = fma(w, gv[m], acc[m]);
          }
#pragma unroll
        for (int m = 0; m < 6; m++) ddg[sym(a, b)][m] = acc[m] * i144h2;
      }
  }
  double gu[6];
  {
    const double c00 = g0[3] * g0[5] - g0[4] * g0[4];
    const double c01 = g0[2] * g0[4] - g0[1] * g0[5];
    const double c02 = g0[1] * g0[4] - g0[2] * g0[3];
    const double det = g0[0] * c00 + g0[1] * c01 + g0[2] * c02;
    const double idet = 1.0 / det;
    gu[0] = c00 * idet;
    gu[1] = c01 * idet;
    gu[2] = c02 * idet;
    gu[3] = (g0[0] * g0[5] - g0[2] * g0[2]) * idet;
    gu[4] = (g0[1] * g0[2] - g0[0] * g0[4]) * idet;
    gu[5] = (g0[0] * g0[3] - g0[1] * g0[1]) * idet;
  }
  // Christoffel symbols: first kind G1[k][ij] = Gamma_kij, second G2[k][ij] =
  // Gamma^k_ij; Ricci tensor (ricci3.cuh)
  double G1[3][6], G2[3][6], Ric[6];
  christoffel3(gu, dg, G1, G2);
  ricci3(gu, ddg, G1, G2, Ric);
  // fiducial triad, orthonormal in g
  double rv[3] = {x[0], x[1], x[2]};
  double pv[3] = {-x[1], x[0], 0.0};
  double tv[3];
  {
    double gu3[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) gu3[a][b] = gu[sym(a, b)];
    const double c00 = g0[3] * g0[5] - g0[4] * g0[4];
    const double c01 = g0[2] * g0[4] - g0[1] * g0[5];
    const double c02 = g0[1] * g0[4] - g0[2] * g0[3];
    const double sdet = sqrt(g0[0] * c00 + g0[1] * c01 + g0[2] * c02);
    const double cr[3] = {pv[1] * rv[2] - pv[2] * rv[1], pv[2] * rv[0] - pv[0] * rv[2],
                          pv[0] * rv[1] - pv[1] * rv[0]};  // eps_klm phi^l r^m
#pragma unroll
    for (int a = 0; a < 3; a++) tv[a] = sdet * (gu3[a][0] * cr[0] + gu3[a][1] * cr[1] + gu3[a][2] * cr[2]);
  }
  const double pp = bil(g0, pv, pv);
  if (!(pp > 0.0)) {
    out[0] = out[1] = 0.0;
    return;
  }
  {
    const double ip = 1.0 / sqrt(pp);
#pragma unroll
    for (int a = 0; a < 3; a++) pv[a] *= ip;
    const double rp = bil(g0, rv, pv);
#pragma unroll
    for (int a = 0; a < 3; a++) rv[a] -= rp * pv[a];
    const double ir = 1.0 / sqrt(bil(g0, rv, rv));
#pragma unroll
    for (int a = 0; a < 3; a++) rv[a] *= ir;
    const double tp = bil(g0, tv, pv), tr = bil(g0, tv, rv);
#pragma unroll
    for (int a = 0; a < 3; a++) tv[a] -= tp * pv[a] + tr * rv[a];
    const double it = 1.0 / sqrt(bil(g0, tv, tv));
#pragma unroll
    for (int a = 0; a < 3; a++) tv[a] *= it;
  }
  // forms on the triad (t = theta, p = phi, r); mb = (t - i p)/sqrt2, n = -r/sqrt2
  const double Rtt = bil(Ric, tv, tv), Rpp = bil(Ric, pv, pv), Rtp = bil(Ric, tv, pv);
  const double Ktt = bil(k0, tv, tv), Kpp = bil(k0, pv, pv), Ktp = bil(k0, tv, pv);
  const double Krr = bil(k0, rv, rv), Krt = bil(k0, rv, tv), Krp = bil(k0, rv, pv);
  double trK = 0.0;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) trK = fma(gu[sym(a, b)], k0[sym(a, b)], trK);
  // (K.K)(a, b) = (K a)_m g^mn (K b)_n
  double Kt[3], Kp[3];
#pragma unroll
  for (int m = 0; m < 3; m++) {
    Kt[m] = k0[sym(m, 0)] * tv[0] + k0[sym(m, 1)] * tv[1] + k0[sym(m, 2)] * tv[2];
    Kp[m] = k0[sym(m, 0)] * pv[0] + k0[sym(m, 1)] * pv[1] + k0[sym(m, 2)] * pv[2];
  }
  const double KKtt = bil(gu, Kt, Kt), KKpp = bil(gu, Kp, Kp), KKtp = bil(gu, Kt, Kp);
  // T(c; a, b) = c^k D_k K(a, b) = c^k [a^j b^l d_k K_jl - K(Gamma_k a, b) - K(a, Gamma_k b)]
  auto T = [&](const double c[3], const double a[3], const double b[3]) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      double Ga[3], Gb[3];
#pragma unroll
      for (int m = 0; m < 3; m++) {
        Ga[m] = G2[m][sym(k, 0)] * a[0] + G2[m][sym(k, 1)] * a[1] + G2[m][sym(k, 2)] * a[2];
        Gb[m] = G2[m][sym(k, 0)] * b[0] + G2[m][sym(k, 1)] * b[1] + G2[m][sym(k, 2)] * b[2];
      }
      s = fma(c[k], bil(dk[k], a, b) - bil(k0, Ga, b) - bil(k0, a, Gb), s);
    }
    return s;
  };
  const double Trtt = T(rv, tv, tv), Trpp = T(rv, pv, pv), Trtp = T(rv, tv, pv);
  const double Tttr = T(tv, tv, rv), Tppr = T(pv, pv, rv), Tptr = T(pv, tv, rv), Ttpr = T(tv, pv, rv);
  // complex pieces (re, im)
  const double Rmm_re = 0.5 * (Rtt - Rpp), Rmm_im = -Rtp;                     // R(mb,mb)
  const double Kmm_re = 0.5 * (Ktt - Kpp), Kmm_im = -Ktp;                     // K(mb,mb)
  const double Knn = 0.5 * Krr;                                               // K(n,n)
  const double Knm_re = -0.5 * Krt, Knm_im = 0.5 * Krp;                       // K(n,mb)
  const double KKmm_re = 0.5 * (KKtt - KKpp), KKmm_im = -KKtp;                // (K.K)(mb,mb)
  const double s2 = 0.70710678118654752440;                                   // 1/sqrt2
  // n^k D_k K(mb,mb) = -(1/sqrt2)(1/2)[T(r;t,t) - T(r;p,p) - 2i T(r;t,p)]
  const double A_re = -s2 * 0.5 * (Trtt - Trpp), A_im = s2 * Trtp;
  // mb^l D_l K(mb,n) = -(1/(2 sqrt2))[T(t;t,r) - T(p;p,r) - i (T(p;t,r) + T(t;p,r))]
  const double B_re = -0.5 * s2 * (Tttr - Tppr), B_im = 0.5 * s2 * (Tptr + Ttpr);
  const double sq2 = 1.41421356237309504880;
  double re = Rmm_re + Knn * Kmm_re - (Knm_re * Knm_re - Knm_im * Knm_im) + sq2 * (A_re - B_re) +
              0.5 * (trK * Kmm_re - KKmm_re);
  double im = Rmm_im + Knn * Kmm_im - 2.0 * Knm_re * Knm_im + sq2 * (A_im - B_im) + 0.5 * (trK * Kmm_im - KKmm_im);
  out[0] = re;
  out[1] = im;
}

template <bool PRE>
__global__ void __launch_bounds__(PB) psi4_kernel(Grid g, const double* __restrict__ y,
                                                  const double* __restrict__ adm, double* __restrict__ out) {
  const long long npts = (long long)g.n0 * g.n1 * g.n2;
  const long long tid = (long long)blockIdx.x * PB + threadIdx.x;
  if (tid >= npts) return;
  const int ii = (int)(tid % g.n0);
  const int jj = (int)((tid / g.n0) % g.n1);
  const int kk = (int)(tid / ((long long)g.n0 * g.n1));
  const long long id = lin(g, ii + GH, jj + GH, kk + GH);
  const double x[3] = {cell_coord(g.xmin0, ii, g.h), cell_coord(g.xmin1, jj, g.h), cell_coord(g.xmin2, kk, g.h)};
  double o[2];
  psi4_point<PRE>(g, y, adm, id, x, o);
  out[id] = o[0];
  out[g.fstride + id] = o[1];
}

}  // namespace

cudaError_t launch_psi4(const Grid& g, const double* y, double* out, cudaStream_t s, double* adm_scratch) {
  const long long npts = (long long)g.n0 * g.n1 * g.n2;
  const unsigned blocks = (unsigned)((npts + PB - 1) / PB);
  if (adm_scratch) {
    cudaError_t e = launch_adm_fields(g, y, adm_scratch, s);
    if (e != cudaSuccess) return e;
    psi4_kernel<true><<<blocks, PB, 0, s>>>(g, y, adm_scratch, out);
  } else {
    psi4_kernel<false><<<blocks, PB, 0, s>>>(g, y, nullptr, out);
  }
  return cudaGetLastError();
}

}  // namespace bssn
