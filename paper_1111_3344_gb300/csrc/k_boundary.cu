// Outer boundary: Sommerfeld radiative condition (arXiv:1111.3344, Sec.
// "Boundary Conditions") and periodic ghost copies.
//
// Sommerfeld: at each ghost point b the radiative part is
//   rad = -v0 (x^i / r) d_i X - v0 (X - X0) / r
// with second-order derivatives (centred where both neighbours are stored,
// one-sided inward on the outermost layer), plus the p = 2 power-law
// correction taken from the inner neighbour j = b - n (n the sum of the
// outward normals of the faces b lies beyond), layer by layer from the
// innermost outwards: rhs_b = rad_b + (r_j / r_b)^2 (rhs_j - rad_j).
// Unrolled along the chain b -> j -> ... -> a (a the first interior point)
// the factors telescope to
//   rhs_b = rad_b + (r_a / r_b)^2 (rhs_a - rad_a),
// so each ghost point is independent: one thread per ghost point, no layer
// ordering.  X0 = 1 for alpha, W and the diagonal of gt, else 0; v0 = sqrt 2
// for alpha and K, else 1.  The boundary arithmetic is float64 on both paths.
#include "bssn_internal.cuh"

namespace bssn {

__device__ __forceinline__ void x0v0(const Grid& g, int f, double& X0, double& v0) {
  X0 = 0.0;
  v0 = 1.0;
  if (f == F_ALP || (f == F_CHI && g.use_w) || f == F_GT + 0 || f == F_GT + 3 || f == F_GT + 5)
    X0 = 1.0;
  if (f == F_ALP || f == F_TRK) v0 = 1.4142135623730951;
}

__device__ __forceinline__ double coordv(const Grid& g, int d, int i) {
  const double xm = d == 0 ? g.xmin0 : (d == 1 ? g.xmin1 : g.xmin2);
  return xm + (i - GH + 0.5) * g.h;
}

// Radiative right-hand side of field f at stored point I; p points at the
// field's value there (float64 or float storage).
template <typename S>
__device__ double rad_at(const Grid& g, const S* __restrict__ p, int f, const int I[3],
                         const double x[3], double r) {
  const long long sd[3] = {1, g.pitch, g.plane};
  const int dims[3] = {g.sx, g.sy, g.sz};
  double X0, v0;
  x0v0(g, f, X0, v0);
  const double i2h = 0.5 / g.h;
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const long long q = sd[d];
    double der;
    if (I[d] >= 1 && I[d] + 1 < dims[d])
      der = ((double)p[q] - (double)p[-q]) * i2h;
    else if (I[d] + 1 >= dims[d])
      der = (3.0 * (double)p[0] - 4.0 * (double)p[-q] + (double)p[-2 * q]) * i2h;
    else
      der = -(3.0 * (double)p[0] - 4.0 * (double)p[q] + (double)p[2 * q]) * i2h;
    s = fma(x[d] / r, der, s);
  }
  return -v0 * s - v0 * ((double)p[0] - X0) / r;
}

template <typename S>
__global__ void sommerfeld_kernel(Grid g, StageArgsT<S> a, const S* __restrict__ kanchor) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)g.sx * g.sy * g.sz;
  if (tid >= total) return;
  int I[3];
  I[0] = (int)(tid % g.sx);
  I[1] = (int)((tid / g.sx) % g.sy);
  I[2] = (int)(tid / ((long long)g.sx * g.sy));
  const int n[3] = {g.n0, g.n1, g.n2};
  bool ghost = false;
#pragma unroll
  for (int d = 0; d < 3; d++) ghost |= (I[d] < GH || I[d] >= GH + n[d]);
  if (!ghost) return;
  // walk to the anchor: each step moves one layer inward along the summed normal
  int A[3] = {I[0], I[1], I[2]};
  for (int step = 0; step < GH; step++) {
    bool moved = false;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      if (A[d] < GH) { A[d] += 1; moved = true; }
      else if (A[d] >= GH + n[d]) { A[d] -= 1; moved = true; }
    }
    if (!moved) break;
  }
  double xb[3], xa[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    xb[d] = coordv(g, d, I[d]);
    xa[d] = coordv(g, d, A[d]);
  }
  const double rb = sqrt(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2]);
  const double ra = sqrt(xa[0] * xa[0] + xa[1] * xa[1] + xa[2] * xa[2]);
  const double fac = (ra / rb) * (ra / rb);
  const long long ib = lin(g, I[0], I[1], I[2]);
  const long long ia = lin(g, A[0], A[1], A[2]);
  const long long fs = g.fstride;
  const int nf = g.shift == BSSN_SHIFT_FROZEN ? F_BETA : NF;
  for (int f = 0; f < NF; f++) {
    double rhs = 0.0;
    if (f < nf) {
      double radb, rada;
      if (f == F_CHI && a.srcw) {
        radb = rad_at<double>(g, a.srcw + ib, f, I, xb, rb);
        rada = rad_at<double>(g, a.srcw + ia, f, A, xa, ra);
      } else {
        radb = rad_at<S>(g, a.src + f * fs + ib, f, I, xb, rb);
        rada = rad_at<S>(g, a.src + f * fs + ia, f, A, xa, ra);
      }
      const double ka = (a.mode == MODE_RHS) ? a.rhs[f * fs + ia] : (double)kanchor[f * fs + ia];
      rhs = fma(fac, ka - rada, radb);
    }
    const long long o = f * fs + ib;
    if (a.mode == MODE_RHS) {
      a.rhs[o] = rhs;
    } else if (a.mode == MODE_LAST) {
      const double v = fma(a.b_dt, rhs, a.acc[o]);
      a.acc[o] = v;
      if (a.out0) a.out0[o] = (S)v;
      if (f == F_CHI && a.out0w) a.out0w[ib] = v;
    } else {
      const double y = a.yn[o];
      const double v = fma(a.a_dt, rhs, y);
      a.out0[o] = (S)v;
      if (f == F_CHI && a.out0w) a.out0w[ib] = v;
      a.acc[o] = fma(a.b_dt, rhs, a.mode == MODE_FIRST ? y : a.acc[o]);
    }
  }
}

template <typename S>
static cudaError_t launch_sommerfeld_t(const Grid& g, const StageArgsT<S>& a, const S* kanchor,
                                       cudaStream_t s) {
  const long long total = (long long)g.sx * g.sy * g.sz;
  const int bs = 256;
  sommerfeld_kernel<S><<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(g, a, kanchor);
  return cudaGetLastError();
}

cudaError_t launch_sommerfeld(const Grid& g, const StageArgs& a, const double* kanchor,
                              cudaStream_t s) {
  return launch_sommerfeld_t<double>(g, a, kanchor, s);
}
cudaError_t launch_sommerfeld_mixed(const Grid& g, const StageArgsMixed& a, const float* kanchor,
                                    cudaStream_t s) {
  return launch_sommerfeld_t<float>(g, a, kanchor, s);
}

// Periodic ghosts: copy from the wrapped interior point, all fields (and the
// float64 W array of a mixed stage buffer when w is non-null).
template <typename S>
__global__ void periodic_fill_kernel(Grid g, S* __restrict__ y, double* __restrict__ w) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)g.sx * g.sy * g.sz;
  if (tid >= total) return;
  const int i = (int)(tid % g.sx);
  const int j = (int)((tid / g.sx) % g.sy);
  const int k = (int)(tid / ((long long)g.sx * g.sy));
  const bool ghost = i < GH || i >= GH + g.n0 || j < GH || j >= GH + g.n1 || k < GH ||
                     k >= GH + g.n2;
  if (!ghost) return;
  const int si = GH + ((i - GH) % g.n0 + g.n0) % g.n0;
  const int sj = GH + ((j - GH) % g.n1 + g.n1) % g.n1;
  const int sk = GH + ((k - GH) % g.n2 + g.n2) % g.n2;
  const long long d = lin(g, i, j, k), s = lin(g, si, sj, sk);
  for (int f = 0; f < NF; f++) y[f * g.fstride + d] = y[f * g.fstride + s];
  if (w) w[d] = w[s];
}

cudaError_t launch_periodic_fill(const Grid& g, double* y, cudaStream_t s) {
  const long long total = (long long)g.sx * g.sy * g.sz;
  const int bs = 256;
  periodic_fill_kernel<double><<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(g, y, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_periodic_fill_mixed(const Grid& g, float* y, double* w, cudaStream_t s) {
  const long long total = (long long)g.sx * g.sy * g.sz;
  const int bs = 256;
  periodic_fill_kernel<float><<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(g, y, w);
  return cudaGetLastError();
}

}  // namespace bssn
