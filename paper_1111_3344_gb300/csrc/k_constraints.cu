// Hamiltonian and momentum constraints with deterministic norm reductions
// (arXiv:1111.3344, Sec. "Other analysis modules"): H = R - K^i_j K^j_i + K^2,
// M_i = nabla_j K_i^j - nabla_i K in vacuum, from the ADM fields
// gamma_ij = e^{4 phi} gt_ij and K_ij = e^{4 phi}(At_ij + gt_ij K / 3), which
// are formed pointwise at every stencil point on the fly (no scratch grids),
// then differenced with the same 4th-order stencils as the evolution.
//   R_ij = 1/2 gamma^kl (d_k d_j g_il + d_i d_l g_kj - d_k d_l g_ij - d_i d_j g_kl)
//          + gamma^kl (Gamma^m_il Gamma_mkj - Gamma^m_ij Gamma_mkl)
//   M_i  = gamma^jk (d_k K_ij - d_i K_jk) - Gamma^l K_il + Gamma^l_ij K_l^j
// (the Christoffel terms of gamma^jk (nabla_k K_ij - nabla_i K_jk) after the
// symmetric pair cancels).  With a stress-energy tensor, H gets -16 pi E and
// M_i gets -8 pi S_i.  Float64 in every precision mode.
//
// Reduction: one thread per interior point; per block a warp-shuffle tree in
// each warp and a shuffle tree over the warp results, in a fixed order, into
// per-block partials (8 sums of squares, 8 maxima, 2 counts); then one block
// folds the partials the same way: the result does not depend on scheduling.
#include "bssn_internal.cuh"
#include "ricci3.cuh"

namespace bssn {

// max that lets a NaN through (so a blown-up state shows in the Linf norms)
__device__ __forceinline__ double nanmax(double a, double b) { return (b > a || b != b) ? b : a; }

constexpr int CB = 256;   // threads per block
constexpr int NPART = 18; // partial values per block

// ADM fields at one stored point, formed from the state (PRE = false) or read
// from a buffer of 12 fields gamma_ij, K_ij filled by adm_fields_kernel with
// the same operations (PRE = true), so both give the same bits.
template <bool PRE>
__device__ __forceinline__ void adm_at(const Grid& g, const double* __restrict__ y,
                                       const double* __restrict__ adm, long long id, double gam[6],
                                       double K[6], bool needK) {
  const long long fs = g.fstride;
  if constexpr (PRE) {
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

template <bool PRE>
__device__ void constraints_point(const Grid& g, const double* __restrict__ y,
                                  const double* __restrict__ adm, long long id, double out[4]) {
  const long long sd[3] = {1, g.pitch, g.plane};
  const double i12h = g.i12h;
  const double i12h2 = g.i12h2;
  const double i144h2 = g.i144h2;
  double g0[6], k0[6];
  adm_at<PRE>(g, y, adm, id, g0, k0, true);
  double dg[3][6], dk[3][6], ddg[6][6];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    double gp1[6], gm1[6], gp2[6], gm2[6], kp1[6], km1[6], kp2[6], km2[6];
    adm_at<PRE>(g, y, adm, id + sd[d], gp1, kp1, true);
    adm_at<PRE>(g, y, adm, id - sd[d], gm1, km1, true);
    adm_at<PRE>(g, y, adm, id + 2 * sd[d], gp2, kp2, true);
    adm_at<PRE>(g, y, adm, id - 2 * sd[d], gm2, km2, true);
#pragma unroll
    for (int m = 0; m < 6; m++) {
      dg[d][m] = fma(8.0, gp1[m] - gm1[m], -(gp2[m] - gm2[m])) * i12h;
      dk[d][m] = fma(8.0, kp1[m] - km1[m], -(kp2[m] - km2[m])) * i12h;
      ddg[sym(d, d)][m] = fma(-30.0, g0[m], fma(16.0, gp1[m] + gm1[m], -(gp2[m] + gm2[m]))) * i12h2;
    }
  }
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
          adm_at<PRE>(g, y, adm, id + off[p] * sd[a] + off[q] * sd[b], gv, dummy, false);
          const double w = c[p] * c[q];
#pragma unroll
          for (int m = 0; m < 6; m++) acc[m] = fma(w, gv[m], acc[m]);
        }
#pragma unroll
      for (int m = 0; m < 6; m++) ddg[sym(a, b)][m] = acc[m] * i144h2;
    }

  // inverse metric
  double gu[6];
  {
    const double c00 = g0[3] * g0[5] - g0[4] * g0[4];
    const double c01 = g0[2] * g0[4] - g0[1] * g0[5];
    const double c02 = g0[1] * g0[4] - g0[2] * g0[3];
    const double idet = 1.0 / (g0[0] * c00 + g0[1] * c01 + g0[2] * c02);
    gu[0] = c00 * idet;
    gu[1] = c01 * idet;
    gu[2] = c02 * idet;
    gu[3] = (g0[0] * g0[5] - g0[2] * g0[2]) * idet;
    gu[4] = (g0[1] * g0[2] - g0[0] * g0[4]) * idet;
    gu[5] = (g0[0] * g0[3] - g0[1] * g0[1]) * idet;
  }
  // Christoffel symbols and Ricci tensor (ricci3.cuh); R = g^ij R_ij
  double G1[3][6], G2[3][6], Ric[6];
  christoffel3(gu, dg, G1, G2);
  ricci3(gu, ddg, G1, G2, Ric);
  double R = 0.0;
#pragma unroll
  for (int m = 0; m < 6; m++) R = fma((m == 0 || m == 3 || m == 5) ? gu[m] : 2.0 * gu[m], Ric[m], R);
  double Kud[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      Kud[a][b] = gu[sym(a, 0)] * k0[sym(0, b)] + gu[sym(a, 1)] * k0[sym(1, b)] +
                  gu[sym(a, 2)] * k0[sym(2, b)];
  const double trK = Kud[0][0] + Kud[1][1] + Kud[2][2];
  double KK = 0.0;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) KK = fma(Kud[a][b], Kud[b][a], KK);
  out[0] = R - KK + trK * trK;

  // Gamma^l = gamma^jk Gamma^l_jk
  double Gc[3];
#pragma unroll
  for (int l = 0; l < 3; l++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 3; j++)
#pragma unroll
      for (int k = 0; k < 3; k++) s = fma(gu[sym(j, k)], G2[l][sym(j, k)], s);
    Gc[l] = s;
  }
#pragma unroll
  for (int i = 0; i < 3; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 3; j++)
#pragma unroll
      for (int k = 0; k < 3; k++) s = fma(gu[sym(j, k)], dk[k][sym(i, j)] - dk[i][sym(j, k)], s);
#pragma unroll
    for (int l = 0; l < 3; l++) {
      s = fma(-Gc[l], k0[sym(i, l)], s);
      // Gamma^l_ij K_l^j with K_l^j = Kud[j][l] (K symmetric)
#pragma unroll
      for (int j = 0; j < 3; j++) s = fma(G2[l][sym(i, j)], Kud[j][l], s);
    }
    out[1 + i] = s;
  }
  if (g.tmunu) {
    // matter: H -= 16 pi E, M_i -= 8 pi S_i
    const long long fs = g.fstride;
    const double alp = __ldg(y + F_ALP * fs + id);
    const double beta[3] = {__ldg(y + F_BETA * fs + id), __ldg(y + (F_BETA + 1) * fs + id),
                            __ldg(y + (F_BETA + 2) * fs + id)};
    double E, Si[3], Sij[6];
    matter_at<double>(g, id, alp, beta, E, Si, Sij);
    out[0] -= 16.0 * M_PI * E;
#pragma unroll
    for (int q = 0; q < 3; q++) out[1 + q] -= 8.0 * M_PI * Si[q];
  }
}

// Combine rule of partial slot q: max (NaN-propagating) for the Linf slots,
// sum for the rest.
__device__ __forceinline__ bool is_max_slot(int q) { return (q >= 4 && q < 8) || (q >= 12 && q < 16); }
__device__ __forceinline__ double combine(int q, double a, double b) {
  return is_max_slot(q) ? nanmax(a, b) : a + b;
}

// Block reduction of NPART values per thread in a fixed order: a shuffle tree
// inside each warp (offsets 16, 8, 4, 2, 1), the warp results through shared
// memory, then the same shuffle tree over them in warp 0.  Thread 0 returns
// the block's values in v.
__device__ __forceinline__ void block_reduce(double v[NPART]) {
  __shared__ double wsum[NPART][CB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < NPART; q++) v[q] = combine(q, v[q], __shfl_down_sync(0xffffffffu, v[q], off));
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NPART; q++) wsum[q][warp] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NPART; q++) v[q] = lane < CB / 32 ? wsum[q][lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < NPART; q++) v[q] = combine(q, v[q], __shfl_down_sync(0xffffffffu, v[q], off));
  }
}

template <bool PRE>
__global__ void __launch_bounds__(CB) constraints_kernel(Grid g, const double* __restrict__ y,
                                                         const double* __restrict__ adm, Punct pu,
                                                         double* __restrict__ partials) {
  const long long npts = (long long)g.n0 * g.n1 * g.n2;
  const long long tid = (long long)blockIdx.x * CB + threadIdx.x;
  double v[NPART];
#pragma unroll
  for (int q = 0; q < NPART; q++) v[q] = 0.0;
  if (tid < npts) {
    const int ii = (int)(tid % g.n0);
    const int jj = (int)((tid / g.n0) % g.n1);
    const int kk = (int)(tid / ((long long)g.n0 * g.n1));
    const int i = ii + GH, j = jj + GH, k = kk + GH;
    double c4[4];
    constraints_point<PRE>(g, y, adm, lin(g, i, j, k), c4);
    const double x = cell_coord(g.xmin0, ii, g.h);
    const double yy = cell_coord(g.xmin1, jj, g.h);
    const double z = cell_coord(g.xmin2, kk, g.h);
    bool outside = true;
    for (int a = 0; a < pu.n; a++) {
      const double dx = x - pu.p[a][1], dy = yy - pu.p[a][2], dz = z - pu.p[a][3];
      if (sqrt(dx * dx + dy * dy + dz * dz) <= pu.r_ex) outside = false;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const double sq = c4[q] * c4[q], ab = fabs(c4[q]);
      v[q] = sq;
      v[4 + q] = ab;
      v[8 + q] = outside ? sq : 0.0;
      v[12 + q] = outside ? ab : 0.0;
    }
    v[16] = 1.0;
    v[17] = outside ? 1.0 : 0.0;
  }
  block_reduce(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NPART; q++) partials[(long long)blockIdx.x * NPART + q] = v[q];
}

__global__ void __launch_bounds__(CB) constraints_finalize(const double* __restrict__ partials,
                                                           int nblocks, double* __restrict__ out) {
  double v[NPART];
#pragma unroll
  for (int q = 0; q < NPART; q++) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += CB) {
#pragma unroll
    for (int q = 0; q < NPART; q++) v[q] = combine(q, v[q], partials[(long long)b * NPART + q]);
  }
  block_reduce(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 16; q++) {
      const int set = q / 8, within = q % 8;
      const double cnt = v[16 + set];
      out[q] = within < 4 ? (cnt > 0.0 ? sqrt(v[set * 8 + within] / cnt) : 0.0) : v[set * 8 + within];
    }
  }
}

int constraints_blocks(const Grid& g) {
  const long long npts = (long long)g.n0 * g.n1 * g.n2;
  return (int)((npts + CB - 1) / CB);
}

// gamma_ij = e^{4 phi} gt_ij and K_ij = e^{4 phi}(At_ij + gt_ij K/3) at every
// stored point into adm (12 fields of the register layout), with the
// operations of adm_at<false>.
__global__ void adm_fields_kernel(Grid g, const double* __restrict__ y, double* __restrict__ adm) {
  const long long n = g.fstride;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    double gam[6], K[6];
    adm_at<false>(g, y, nullptr, id, gam, K, true);
#pragma unroll
    for (int m = 0; m < 6; m++) {
      adm[m * n + id] = gam[m];
      adm[(6 + m) * n + id] = K[m];
    }
  }
}

cudaError_t launch_adm_fields(const Grid& g, const double* y, double* adm, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  adm_fields_kernel<<<sms * 8, 256, 0, s>>>(g, y, adm);
  return cudaGetLastError();
}

cudaError_t launch_constraints(const Grid& g, const double* y, const double* punct4, int npunct,
                               double r_excise, double* partials, int nblocks, double* dout16,
                               cudaStream_t s, double* adm_scratch) {
  Punct pu{};
  pu.n = npunct < 8 ? npunct : 8;
  for (int a = 0; a < pu.n; a++)
    for (int q = 0; q < 4; q++) pu.p[a][q] = punct4[4 * a + q];
  pu.r_ex = r_excise;
  cudaError_t e;
  if (adm_scratch) {
    if ((e = launch_adm_fields(g, y, adm_scratch, s)) != cudaSuccess) return e;
    constraints_kernel<true><<<nblocks, CB, 0, s>>>(g, y, adm_scratch, pu, partials);
  } else {
    constraints_kernel<false><<<nblocks, CB, 0, s>>>(g, y, nullptr, pu, partials);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  constraints_finalize<<<1, CB, 0, s>>>(partials, nblocks, dout16);
  return cudaGetLastError();
}

}  // namespace bssn
