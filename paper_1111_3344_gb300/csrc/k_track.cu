// Puncture tracking (arXiv:1111.3344, Sec. "Object tracking"): every
// puncture moves by dx^i/dt = -beta^i at its position, one forward-Euler step
// per RK4 step with the shift of y_n (the state at the start of the step):
//   x_{n+1} = x_n - dt beta^i(t_n, x_n).
// The shift is interpolated by the tensor product of 4-point Lagrange
// polynomials (cubic in each direction) on stored points i0-1 .. i0+2, i0 the
// stored point at or below the position; near the edge of the stored block
// the stencil is shifted inward (the polynomial then extrapolates), so every
// read stays inside the block whatever the position (NaN included).
//
// Positions live in device memory as rows {m, x, y, z}, so the step needs no
// host round trip; one thread per puncture.
#include "bssn_internal.cuh"

namespace bssn {

namespace {

__device__ __forceinline__ double lagrange4(int m, double u) {
  double v = 1.0;
#pragma unroll
  for (int n = -1; n <= 2; n++)
    if (n != m) v *= (u - n) / (double)(m - n);
  return v;
}

__device__ __forceinline__ void interp_setup(double x, double xmin, double h, int stored, int& i0, double& u) {
  // stored point 0 sits at xmin + (0 - GH + 1/2) h
  const double s = (x - (xmin + (0.5 - GH) * h)) / h;
  const double fl = floor(s);
  int b = (fl >= 1.0 && fl <= (double)(stored - 3)) ? (int)fl : (fl > 1.0 ? stored - 3 : 1);
  i0 = b;
  u = s - b;
}

__global__ void track_kernel(Grid g, const double* __restrict__ y, double* __restrict__ punct, int np,
                             double dt) {
  const int a = threadIdx.x;
  if (a >= np) return;
  double* p = punct + 4 * a;
  const double xyz[3] = {p[1], p[2], p[3]};
  int i0[3];
  double u[3];
  interp_setup(xyz[0], g.xmin0, g.h, g.sx, i0[0], u[0]);
  interp_setup(xyz[1], g.xmin1, g.h, g.sy, i0[1], u[1]);
  interp_setup(xyz[2], g.xmin2, g.h, g.sz, i0[2], u[2]);
  double l[3][4];
#pragma unroll
  for (int d = 0; d < 3; d++)
#pragma unroll
    for (int m = 0; m < 4; m++) l[d][m] = lagrange4(m - 1, u[d]);
  double beta[3] = {0.0, 0.0, 0.0};
  for (int mk = 0; mk < 4; mk++)
    for (int mj = 0; mj < 4; mj++) {
      const double wjk = l[1][mj] * l[2][mk];
      const long long row = lin(g, i0[0] - 1, i0[1] - 1 + mj, i0[2] - 1 + mk);
#pragma unroll
      for (int mi = 0; mi < 4; mi++) {
        const double w = l[0][mi] * wjk;
#pragma unroll
        for (int d = 0; d < 3; d++) beta[d] = fma(w, __ldg(y + (F_BETA + d) * g.fstride + row + mi), beta[d]);
      }
    }
#pragma unroll
  for (int d = 0; d < 3; d++) p[1 + d] = xyz[d] - dt * beta[d];
}

}  // namespace

cudaError_t launch_track(const Grid& g, const double* y, double* dpunct, int np, double dt, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  track_kernel<<<1, 32, 0, s>>>(g, y, dpunct, np, dt);
  return cudaGetLastError();
}

}  // namespace bssn
