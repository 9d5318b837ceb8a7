// General initial data: ADM fields -> BSSN variables on the device (arXiv:
// 1111.3344, Sec. "Initial Conditions": the BSSN quantities from their
// definitions with B^i = 0; Gt^i from derivatives of the metric inside the
// grid and by cubic extrapolation on the outer layers -- faces perpendicular,
// edges and corners along the summed normals, innermost layer first).
//
//   phi = ln(det gamma) / 12, W = det^{-1/6}, gt = det^{-1/3} gamma,
//   K = gamma^ij K_ij, At = det^{-1/3} (K_ij - gamma_ij K / 3),
//   Gt^i = gt^{jk} gt^{il} Gt_ljk with 4th-order first derivatives of gt,
//   ghost layer L (L = 1, 2, 3 in order): v(b) = 4 v(b-n) - 6 v(b-2n)
//   + 4 v(b-3n) - v(b-4n), n the summed outward normal of b.
#include "bssn_internal.cuh"
#include "rhs_point.cuh"

namespace bssn {

// In place: y holds the 16 ADM fields in its first 16 field slots (alpha,
// beta^i, gamma_ij, K_ij) and receives the 24 BSSN fields at the same point.
__global__ void adm_convert_kernel(Grid g, double* __restrict__ y) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)g.sx * g.sy * g.sz;
  if (tid >= total) return;
  const int i = (int)(tid % g.sx), j = (int)((tid / g.sx) % g.sy), k = (int)(tid / ((long long)g.sx * g.sy));
  const long long id = lin(g, i, j, k), fs = g.fstride;
  double a[16];
#pragma unroll
  for (int q = 0; q < 16; q++) a[q] = y[q * fs + id];
  const double* gm = a + 4;
  const double* Km = a + 10;
  const double c00 = gm[3] * gm[5] - gm[4] * gm[4];
  const double c01 = gm[2] * gm[4] - gm[1] * gm[5];
  const double c02 = gm[1] * gm[4] - gm[2] * gm[3];
  const double det = gm[0] * c00 + gm[1] * c01 + gm[2] * c02;
  const double idet = 1.0 / det;
  const double gu[6] = {c00 * idet, c01 * idet, c02 * idet, (gm[0] * gm[5] - gm[2] * gm[2]) * idet,
                        (gm[1] * gm[2] - gm[0] * gm[4]) * idet, (gm[0] * gm[3] - gm[1] * gm[1]) * idet};
  double trK = 0.0;
#pragma unroll
  for (int m = 0; m < 6; m++) trK += (m == 0 || m == 3 || m == 5 ? 1.0 : 2.0) * gu[m] * Km[m];
  const double ld = log(det);
  const double em4 = exp(-ld / 3.0);
  double out[NF];
  out[F_CHI] = g.use_w ? exp(-ld / 6.0) : ld / 12.0;
#pragma unroll
  for (int m = 0; m < 6; m++) {
    out[F_GT + m] = em4 * gm[m];
    out[F_AT + m] = em4 * (Km[m] - gm[m] * trK / 3.0);
  }
  out[F_TRK] = trK;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    out[F_GAM + d] = 0.0;
    out[F_BETA + d] = a[1 + d];
    out[F_B + d] = 0.0;
  }
  out[F_ALP] = a[0];
#pragma unroll
  for (int f = 0; f < NF; f++) y[f * fs + id] = out[f];
}

// Gt^i = gt^{jk} gt^{il} Gt_ljk at interior points.
__global__ void gt_fd_kernel(Grid g, double* __restrict__ y) {
  const int ii = blockIdx.x * blockDim.x + threadIdx.x;
  const int jj = blockIdx.y * blockDim.y + threadIdx.y;
  const int kk = blockIdx.z;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  const long long id = lin(g, ii + GH, jj + GH, kk + GH), fs = g.fstride;
  const long long sd[3] = {1, g.pitch, g.plane};
  double gt[6], dgt[3][6];
#pragma unroll
  for (int m = 0; m < 6; m++) {
    const double* p = y + (F_GT + m) * fs + id;
    gt[m] = p[0];
#pragma unroll
    for (int d = 0; d < 3; d++) dgt[d][m] = d1u<double, double>(p, sd[d]) * g.i12h;
  }
  const double c00 = gt[3] * gt[5] - gt[4] * gt[4];
  const double c01 = gt[2] * gt[4] - gt[1] * gt[5];
  const double c02 = gt[1] * gt[4] - gt[2] * gt[3];
  const double idet = 1.0 / (gt[0] * c00 + gt[1] * c01 + gt[2] * c02);
  const double gu[6] = {c00 * idet, c01 * idet, c02 * idet, (gt[0] * gt[5] - gt[2] * gt[2]) * idet,
                        (gt[1] * gt[2] - gt[0] * gt[4]) * idet, (gt[0] * gt[3] - gt[1] * gt[1]) * idet};
  double G1[3][6];  // Gt_ljk = (d_j g_lk + d_k g_lj - d_l g_jk) / 2
#pragma unroll
  for (int l = 0; l < 3; l++)
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++)
        G1[l][sym(a, b)] = 0.5 * (dgt[a][sym(l, b)] + dgt[b][sym(l, a)] - dgt[l][sym(a, b)]);
  double c[3];  // gt^{jk} Gt_ljk
#pragma unroll
  for (int l = 0; l < 3; l++) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) s = fma(gu[sym(a, b)], G1[l][sym(a, b)], s);
    c[l] = s;
  }
#pragma unroll
  for (int i = 0; i < 3; i++)
    y[(F_GAM + i) * fs + id] = gu[sym(i, 0)] * c[0] + gu[sym(i, 1)] * c[1] + gu[sym(i, 2)] * c[2];
}

// Cubic extrapolation of Gt^i on ghost layer L.
__global__ void gt_extrap_kernel(Grid g, double* __restrict__ y, int L) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ghost_count(g)) return;
  int I[3];
  ghost_decode(g, q, I[0], I[1], I[2]);
  const int n[3] = {g.n0, g.n1, g.n2};
  int nr[3], layer = 0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int o = 0;
    nr[d] = 0;
    if (I[d] < GH) { o = GH - I[d]; nr[d] = -1; }
    else if (I[d] >= GH + n[d]) { o = I[d] - (GH + n[d]) + 1; nr[d] = 1; }
    layer = o > layer ? o : layer;
  }
  if (layer != L) return;
  const long long fs = g.fstride;
  const long long step = nr[0] + (long long)nr[1] * g.pitch + (long long)nr[2] * g.plane;
  const long long ib = lin(g, I[0], I[1], I[2]);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const double* p = y + (F_GAM + c) * fs + ib;
    y[(F_GAM + c) * fs + ib] = 4.0 * p[-step] - 6.0 * p[-2 * step] + 4.0 * p[-3 * step] - p[-4 * step];
  }
}

cudaError_t launch_adm_to_bssn(const Grid& g, double* y, cudaStream_t s) {
  const long long total = (long long)g.sx * g.sy * g.sz;
  adm_convert_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gt_fd_kernel<<<dim3((g.n0 + 31) / 32, (g.n1 + 7) / 8, g.n2), dim3(32, 8, 1), 0, s>>>(g, y);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (g.periodic) return launch_periodic_fill(g, y, s);
  const unsigned ng = ghost_count(g);
  for (int L = 1; L <= GH; L++) {
    gt_extrap_kernel<<<(ng + 255) / 256, 256, 0, s>>>(g, y, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bssn
