// Fused BSSN right-hand side + RK4 stage combination.
//
// One thread per interior point.  The right-hand side (rhs_point.cuh) is
// evaluated from the stage input register and combined at once with y_n and
// the accumulator, so k is never stored except at the interior points next to
// the outer boundary, whose k the Sommerfeld boundary needs (anchor buffer).
// Classical RK4 with registers y_n, acc and two stage buffers (the method of
// lines that evolves the equations of Sec. "Spacetime Curvature Evolution"):
//   stage 1: s1 = y + dt/2 k1,  acc = y + dt/6 k1
//   stage 2: s2 = y + dt/2 k2,  acc += dt/3 k2
//   stage 3: s1 = y + dt k3,    acc += dt/3 k3
//   stage 4: acc += dt/6 k4,    y_{n+1} = acc
//
// Float64 path: everything in double.  Mixed path: stage buffers hold float
// (plus W in double), the stencils and the right-hand side run in float, and
// y_n, acc and the stage combination stay in double.  Where W is below the
// threshold (near a puncture) the W right-hand side is recomputed in double
// from the double W of the stage buffer.
#include "bssn_internal.cuh"
#include "rhs_point.cuh"

namespace bssn {

constexpr int TX = 32, TY = 8;

__device__ __forceinline__ bool on_shell(const Grid& g, int ii, int jj, int kk) {
  return ii == 0 || jj == 0 || kk == 0 || ii == g.n0 - 1 || jj == g.n1 - 1 || kk == g.n2 - 1;
}

__global__ void __launch_bounds__(TX * TY) stage_fp64_kernel(Grid g, StageArgs a) {
  const int ii = blockIdx.x * TX + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  const int i = ii + GH, j = jj + GH, k = kk + GH;
  const long long id = lin(g, i, j, k);
  double r[NF];
  rhs_point<double, double>(g, a.src, id, i, j, k, r);
  const long long fs = g.fstride;
  if (a.mode == MODE_RHS) {
#pragma unroll
    for (int f = 0; f < NF; f++) a.rhs[f * fs + id] = r[f];
    return;
  }
  if (a.kshell && on_shell(g, ii, jj, kk)) {
#pragma unroll
    for (int f = 0; f < NF; f++) a.kshell[f * fs + id] = r[f];
  }
  if (a.mode == MODE_FIRST) {
#pragma unroll
    for (int f = 0; f < NF; f++) {
      const double y = a.yn[f * fs + id];
      a.out0[f * fs + id] = fma(a.a_dt, r[f], y);
      a.acc[f * fs + id] = fma(a.b_dt, r[f], y);
    }
  } else if (a.mode == MODE_MID) {
#pragma unroll
    for (int f = 0; f < NF; f++) {
      const double y = a.yn[f * fs + id];
      a.out0[f * fs + id] = fma(a.a_dt, r[f], y);
      a.acc[f * fs + id] = fma(a.b_dt, r[f], a.acc[f * fs + id]);
    }
  } else {
#pragma unroll
    for (int f = 0; f < NF; f++) a.acc[f * fs + id] = fma(a.b_dt, r[f], a.acc[f * fs + id]);
  }
}

cudaError_t launch_stage_fp64(const Grid& g, const StageArgs& a, cudaStream_t s) {
  dim3 block(TX, TY, 1);
  dim3 grid((g.n0 + TX - 1) / TX, (g.n1 + TY - 1) / TY, g.n2);
  stage_fp64_kernel<<<grid, block, 0, s>>>(g, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- mixed

// W (or phi) right-hand side in float64 from the float64 W of the stage input:
// d_0 W = (W/3)(alpha K - d_k beta^k) (phi: -(alpha/6) K + d_k beta^k / 6),
// plus upwinded advection and KO, as in rhs_point.
__device__ double chi_rhs_fp64(const Grid& g, const float* __restrict__ st,
                               const double* __restrict__ w, long long id) {
  const long long fs = g.fstride;
  const long long sd[3] = {1, g.pitch, g.plane};
  const double i12h = 1.0 / (12.0 * g.h);
  const double chi = w[id];
  const double alp = (double)__ldg(st + F_ALP * fs + id);
  const double trK = (double)__ldg(st + F_TRK * fs + id);
  double beta[3], divb = 0.0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    beta[d] = (double)__ldg(st + (F_BETA + d) * fs + id);
    divb += d1u<double, float>(st + (F_BETA + d) * fs + id, sd[d]) * i12h;
  }
  double r = g.use_w ? (chi * (1.0 / 3.0)) * (alp * trK - divb)
                     : (-1.0 / 6.0) * alp * trK + divb * (1.0 / 6.0);
  Adv up;
  double ab[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    up.s[d] = beta[d] >= 0.0 ? sd[d] : -sd[d];
    ab[d] = fabs(beta[d]);
  }
  double adv, ko;
  adv_ko<double, double>(w + id, sd, up, ab, ab[0] + ab[1] + ab[2], chi, adv, ko);
  return fma(g.ko_eps / (64.0 * g.h), ko, fma(i12h, adv, r));
}

__global__ void __launch_bounds__(TX * TY) stage_mixed_kernel(Grid g, StageArgsMixed a) {
  const int ii = blockIdx.x * TX + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  const int i = ii + GH, j = jj + GH, k = kk + GH;
  const long long id = lin(g, i, j, k);
  float r[NF];
  rhs_point<float, float>(g, a.src, id, i, j, k, r);
  const long long fs = g.fstride;
  // near a puncture the W update runs in float64
  const double w0 = a.srcw[id];
  const double wval = g.use_w ? w0 : exp(-2.0 * w0);
  const double rchi = wval < a.w_thr ? chi_rhs_fp64(g, a.src, a.srcw, id) : (double)r[F_CHI];
  if (a.mode == MODE_RHS) {
    a.rhs[id] = rchi;
#pragma unroll
    for (int f = 1; f < NF; f++) a.rhs[f * fs + id] = (double)r[f];
    return;
  }
  if (a.kshell && on_shell(g, ii, jj, kk)) {
#pragma unroll
    for (int f = 0; f < NF; f++) a.kshell[f * fs + id] = f == F_CHI ? (float)rchi : r[f];
  }
#pragma unroll
  for (int f = 0; f < NF; f++) {
    const double kf = f == F_CHI ? rchi : (double)r[f];
    const long long o = f * fs + id;
    if (a.mode == MODE_LAST) {
      const double v = fma(a.b_dt, kf, a.acc[o]);
      a.acc[o] = v;
      a.out0[o] = (float)v;
      if (f == F_CHI) a.out0w[id] = v;
    } else {
      const double y = a.yn[o];
      const double v = fma(a.a_dt, kf, y);
      a.out0[o] = (float)v;
      if (f == F_CHI) a.out0w[id] = v;
      a.acc[o] = fma(a.b_dt, kf, a.mode == MODE_FIRST ? y : a.acc[o]);
    }
  }
}

cudaError_t launch_stage_mixed(const Grid& g, const StageArgsMixed& a, cudaStream_t s) {
  dim3 block(TX, TY, 1);
  dim3 grid((g.n0 + TX - 1) / TX, (g.n1 + TY - 1) / TY, g.n2);
  stage_mixed_kernel<<<grid, block, 0, s>>>(g, a);
  return cudaGetLastError();
}

// float shadow (and float64 W) of a float64 register, every stored point
__global__ void shadow_kernel(Grid g, const double* __restrict__ y, float* __restrict__ s32,
                              double* __restrict__ w) {
  const long long n = (long long)NF * g.fstride;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double v = y[q];
    s32[q] = (float)v;
    if (q < g.fstride) w[q] = v;
  }
}

cudaError_t launch_shadow(const Grid& g, const double* y, float* s32, double* w, cudaStream_t s) {
  shadow_kernel<<<152 * 8, 256, 0, s>>>(g, y, s32, w);
  return cudaGetLastError();
}

}  // namespace bssn
