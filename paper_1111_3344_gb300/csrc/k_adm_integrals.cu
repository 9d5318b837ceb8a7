// ADM mass and angular momentum as volume integrals (arXiv:1111.3344, Sec.
// "Masses and Momenta", the ML_ADMQuantities form):
//   M   = 1/(16 pi) int [ e^{5 phi}(16 pi E + At_ij At^ij - (2/3) K^2) - e^{phi} Rt ]
//   J_i = 1/(8 pi) eps_ijk int e^{6 phi} [ At^j_k + (2/3) x^j d_k K
//                                          - (1/2) x^j At_ln d_k gt^{ln} + 8 pi x^j S_k ]
// (E = S_k = 0 unless a stress-energy tensor is given)
// with Rt = gt^ij Rt_ij built from the same pieces as the right-hand side
// (the evolved Gt in gt_k(i d_j) Gt^k, d_l gt^{lk} from the metric stencils
// elsewhere), d_k gt^{ln} = -gt^{la} gt^{nb} d_k gt_ab, so that
// At_ln d_k gt^{ln} = -At^{ab} d_k gt_ab; x^j the grid coordinates;
// e^{phi} = W^{-1/2} (W floored) or exp(phi).  The integrals are midpoint
// sums h^3 sum over interior points, over all of them and over the points
// farther than r_excise from every puncture.  Float64 in every precision mode.
//
// One thread per interior point; per block a warp-shuffle tree in each warp
// and over the warp results (fixed order) into 8 partial sums, then one block
// folds the partials the same way, so the result does not depend on
// scheduling.
#include "rhs_point.cuh"
#include "ricci3.cuh"

namespace bssn {

namespace {

constexpr int AB = 256;  // threads per block
constexpr int NQ = 8;    // M, J_x, J_y, J_z; full then excised

__device__ void adm_density(const Grid& g, const double* __restrict__ y, long long id, double x[3],
                            double out[4]) {
  const GlobalAcc<double> acc(g, y, id);
  const double i12h = g.i12h, i12h2 = g.i12h2, i144h2 = g.i144h2;
#define PF(f) acc.ptr(f)
#define SD(f, d) acc.s((f), (d))
  const double chi = __ldg(PF(F_CHI));
  const double trK = __ldg(PF(F_TRK));
  double gt[6], At[6];
#pragma unroll
  for (int m = 0; m < 6; m++) {
    gt[m] = __ldg(PF(F_GT + m));
    At[m] = __ldg(PF(F_AT + m));
  }
  double gu[6];
  {
    const double c00 = gt[3] * gt[5] - gt[4] * gt[4];
    const double c01 = gt[2] * gt[4] - gt[1] * gt[5];
    const double c02 = gt[1] * gt[4] - gt[2] * gt[3];
    const double idet = 1.0 / (gt[0] * c00 + gt[1] * c01 + gt[2] * c02);
    gu[0] = c00 * idet;
    gu[1] = c01 * idet;
    gu[2] = c02 * idet;
    gu[3] = (gt[0] * gt[5] - gt[2] * gt[2]) * idet;
    gu[4] = (gt[1] * gt[2] - gt[0] * gt[4]) * idet;
    gu[5] = (gt[0] * gt[3] - gt[1] * gt[1]) * idet;
  }
  double dgt[3][6], dG[3][3], dK[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
#pragma unroll
    for (int m = 0; m < 6; m++) dgt[d][m] = d1u<double>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, d)) * i12h;
#pragma unroll
    for (int a = 0; a < 3; a++) dG[d][a] = d1u<double>(acc, F_GAM + a, PF(F_GAM + a), SD(F_GAM + a, d)) * i12h;
    dK[d] = d1u<double>(acc, F_TRK, PF(F_TRK), SD(F_TRK, d)) * i12h;
  }
  // -1/2 gt^{kl} d_k d_l gt_ij, accumulated pair by pair
  double Rdd[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int pa = 0; pa < 3; pa++)
#pragma unroll
    for (int pb = pa; pb < 3; pb++) {
      const int pq = sym(pa, pb);
      const double w = (pa == pb) ? -0.5 * gu[pq] : -gu[pq];
#pragma unroll
      for (int m = 0; m < 6; m++) {
        const double dd = (pa == pb)
                              ? d2u<double>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, pa), gt[m]) * i12h2
                              : dmu<double>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, pa), SD(F_GT + m, pb)) * i144h2;
        Rdd[m] = fma(w, dd, Rdd[m]);
      }
    }
#undef PF
#undef SD
  // Christoffel symbols of gt (ricci3.cuh: the terms that cancel left out)
  double G1[3][6], G2[3][6];
  christoffel3(gu, dgt, G1, G2);
  double dgu[3];
  {
    double Tb[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < 3; l++)
#pragma unroll
        for (int a = 0; a < 3; a++) s = fma(gu[sym(l, a)], dgt[l][sym(a, b)], s);
      Tb[b] = s;
    }
#pragma unroll
    for (int kk = 0; kk < 3; kk++)
      dgu[kk] = -(gu[sym(kk, 0)] * Tb[0] + gu[sym(kk, 1)] * Tb[1] + gu[sym(kk, 2)] * Tb[2]);
  }
  // Rt_ij and its trace gt^ij Rt_ij
  double Rtr = 0.0;
  {
    double G1u[3][3][3];
#pragma unroll
    for (int jj = 0; jj < 3; jj++)
#pragma unroll
      for (int kk = 0; kk < 3; kk++)
#pragma unroll
        for (int l = 0; l < 3; l++)
          G1u[jj][kk][l] = gu[sym(l, 0)] * G1[jj][sym(kk, 0)] + gu[sym(l, 1)] * G1[jj][sym(kk, 1)] +
                           gu[sym(l, 2)] * G1[jj][sym(kk, 2)];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++) {
        const int ab = sym(a, b);
        double s = Rdd[ab], t = 0.0;
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
          t = fma(gt[sym(kk, a)], dG[b][kk], t);
          t = fma(gt[sym(kk, b)], dG[a][kk], t);
          t = fma(-dgt[kk][ab], dgu[kk], t);  // Gt_akb + Gt_bka = d_k gt_ab
        }
        s = fma(0.5, t, s);
        if (a == b) {  // the first two quadratic terms coincide
          double q = 0.0;
#pragma unroll
          for (int kk = 0; kk < 3; kk++)
#pragma unroll
            for (int l = 0; l < 3; l++) {
              q = fma(G2[kk][sym(l, a)], G1u[a][kk][l], q);
              s = fma(G2[kk][sym(a, l)], G1u[kk][a][l], s);
            }
          s = fma(2.0, q, s);
        } else {
#pragma unroll
          for (int kk = 0; kk < 3; kk++)
#pragma unroll
            for (int l = 0; l < 3; l++) {
              s = fma(G2[kk][sym(l, a)], G1u[b][kk][l], s);
              s = fma(G2[kk][sym(l, b)], G1u[a][kk][l], s);
              s = fma(G2[kk][sym(a, l)], G1u[kk][b][l], s);
            }
        }
        Rtr = fma(a == b ? gu[ab] : 2.0 * gu[ab], s, Rtr);
      }
  }
  // e^{phi} and its powers
  double ephi;
  if (g.use_w) {
    const double Wd = chi > g.w_floor ? chi : g.w_floor;
    ephi = 1.0 / sqrt(Wd);
  } else {
    ephi = exp(chi);
  }
  const double e2 = ephi * ephi;
  const double e5 = e2 * e2 * ephi;
  const double e6 = e5 * ephi;
  // At^j_k = gt^{jl} At_lk (not symmetric) and At^{ab}
  double Am[3][3], Au[6];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      Am[a][b] = gu[sym(a, 0)] * At[sym(0, b)] + gu[sym(a, 1)] * At[sym(1, b)] + gu[sym(a, 2)] * At[sym(2, b)];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = a; b < 3; b++)
      Au[sym(a, b)] = Am[a][0] * gu[sym(0, b)] + Am[a][1] * gu[sym(1, b)] + Am[a][2] * gu[sym(2, b)];
  double AA = 0.0;
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) AA = fma(At[sym(a, b)], Au[sym(a, b)], AA);
  // matter: E and S_k (zero in vacuum)
  double Em = 0.0, Sk[3] = {0.0, 0.0, 0.0};
  if (g.tmunu) {
    const double alp = __ldg(y + F_ALP * g.fstride + id);
    const double beta[3] = {__ldg(y + F_BETA * g.fstride + id), __ldg(y + (F_BETA + 1) * g.fstride + id),
                            __ldg(y + (F_BETA + 2) * g.fstride + id)};
    double Sij[6];
    matter_at<double>(g, id, alp, beta, Em, Sk, Sij);
  }
  out[0] = (e5 * (16.0 * M_PI * Em + AA - (2.0 / 3.0) * trK * trK) - ephi * Rtr) * (1.0 / (16.0 * M_PI));
  // At_ln d_k gt^{ln} = -At^{ab} d_k gt_ab
  double AdG[3];
#pragma unroll
  for (int kk = 0; kk < 3; kk++) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) s = fma(Au[sym(a, b)], dgt[kk][sym(a, b)], s);
    AdG[kk] = -s;
  }
  double v[3][3];  // v[j][k] = At^j_k + x^j ((2/3) d_k K - (1/2) At_ln d_k gt^{ln})
#pragma unroll
  for (int jj = 0; jj < 3; jj++)
#pragma unroll
    for (int kk = 0; kk < 3; kk++)
      v[jj][kk] = fma(x[jj], (2.0 / 3.0) * dK[kk] - 0.5 * AdG[kk] + 8.0 * M_PI * Sk[kk], Am[jj][kk]);
  const double c = e6 * (1.0 / (8.0 * M_PI));
  out[1] = c * (v[1][2] - v[2][1]);
  out[2] = c * (v[2][0] - v[0][2]);
  out[3] = c * (v[0][1] - v[1][0]);
}

// Fixed-order block sum of NQ values per thread: shuffle tree in each warp,
// then over the warp results in warp 0; thread 0 returns the sums in v.
__device__ __forceinline__ void block_sum(double v[NQ]) {
  __shared__ double wsum[NQ][AB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < NQ; q++) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NQ; q++) wsum[q][warp] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; q++) v[q] = lane < AB / 32 ? wsum[q][lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < NQ; q++) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  }
}

__global__ void __launch_bounds__(AB) adm_integrals_kernel(Grid g, const double* __restrict__ y, Punct pu,
                                                           double* __restrict__ dens,
                                                           double* __restrict__ partials) {
  const long long npts = (long long)g.n0 * g.n1 * g.n2;
  const long long tid = (long long)blockIdx.x * AB + threadIdx.x;
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) v[q] = 0.0;
  if (tid < npts) {
    const int ii = (int)(tid % g.n0);
    const int jj = (int)((tid / g.n0) % g.n1);
    const int kk = (int)(tid / ((long long)g.n0 * g.n1));
    const int i = ii + GH, j = jj + GH, k = kk + GH;
    const long long id = lin(g, i, j, k);
    double x[3] = {cell_coord(g.xmin0, ii, g.h), cell_coord(g.xmin1, jj, g.h), cell_coord(g.xmin2, kk, g.h)};
    double o[4];
    adm_density(g, y, id, x, o);
    if (dens) {
#pragma unroll
      for (int q = 0; q < 4; q++) dens[q * g.fstride + id] = o[q];
    }
    bool outside = true;
    for (int a = 0; a < pu.n; a++) {
      const double dx = x[0] - pu.p[a][1], dy = x[1] - pu.p[a][2], dz = x[2] - pu.p[a][3];
      if (sqrt(dx * dx + dy * dy + dz * dz) <= pu.r_ex) outside = false;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      v[q] = o[q];
      v[4 + q] = outside ? o[q] : 0.0;
    }
  }
  block_sum(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NQ; q++) partials[(long long)blockIdx.x * NQ + q] = v[q];
}

__global__ void __launch_bounds__(AB) adm_integrals_finalize(const double* __restrict__ partials, int nblocks,
                                                             double vol, double* __restrict__ out) {
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; q++) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += AB) {
#pragma unroll
    for (int q = 0; q < NQ; q++) v[q] += partials[(long long)b * NQ + q];
  }
  block_sum(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NQ; q++) out[q] = v[q] * vol;
}

}  // namespace

int adm_integrals_blocks(const Grid& g) {
  const long long npts = (long long)g.n0 * g.n1 * g.n2;
  return (int)((npts + AB - 1) / AB);
}

cudaError_t launch_adm_integrals(const Grid& g, const double* y, const Punct& pu, double* dens,
                                 double* partials, int nblocks, double* dout8, cudaStream_t s) {
  adm_integrals_kernel<<<nblocks, AB, 0, s>>>(g, y, pu, dens, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adm_integrals_finalize<<<1, AB, 0, s>>>(partials, nblocks, g.h * g.h * g.h, dout8);
  return cudaGetLastError();
}

}  // namespace bssn
