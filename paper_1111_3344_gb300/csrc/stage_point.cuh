// Per-point fused stage (right-hand side + RK4 combine), shared by the
// single-grid kernels (k_stage.cu) and the batched persistent kernels
// (k_batch.cu) so that an evolution computes the same bits in either.
#pragma once
#include "bssn_internal.cuh"
#include "rhs_point.cuh"

namespace bssn {

__device__ __forceinline__ bool on_shell(const Grid& g, int ii, int jj, int kk) {
  return ii == 0 || jj == 0 || kk == 0 || ii == g.n0 - 1 || jj == g.n1 - 1 || kk == g.n2 - 1;
}

// Fused stage at interior point (ii, jj, kk) (interior indices), float64.
// XSEG = 32: the calling warp is one full row of 32 x points (see dmx_shfl);
// YROWS > 0: also every thread of the block is inside the grid (D_y D_z
// through shared memory, see rhs_point_acc).
template <int XSEG = 0, int YROWS = 0, int ZS = 1>
__device__ __forceinline__ void stage_point_fp64(const Grid& g, const StageArgs& a, int ii, int jj,
                                                 int kk) {
  const int i = ii + GH, j = jj + GH, k = kk + GH;
  const long long id = lin(g, i, j, k);
  double r[NF];
  rhs_point<double, double, false, XSEG, YROWS, ZS>(g, a.src, id, i, j, k, r);
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
  if (a.mode == MODE_LAST) {
#pragma unroll
    for (int f = 0; f < NF; f++) {
      const long long o = f * fs + id;
      a.yn[o] = fma(a.b_dt, a.ksum[o] + r[f], a.yn[o]);
    }
    return;
  }
#pragma unroll
  for (int f = 0; f < NF; f++) {
    const long long o = f * fs + id;
    a.out0[o] = fma(a.a_dt, r[f], a.src0[o]);
    a.ksum[o] = a.mode == MODE_FIRST ? r[f] : fma(2.0, r[f], a.ksum[o]);
  }
}

// ---------------------------------------------------------------- mixed

// W (or phi) right-hand side in float64 from the float64 W of the stage input:
// d_0 W = (W/3)(alpha K - d_k beta^k) (phi: -(alpha/6) K + d_k beta^k / 6),
// plus upwinded advection and KO, as in rhs_point.
__device__ __forceinline__ double chi_rhs_fp64(const Grid& g, const float* __restrict__ st,
                               const double* __restrict__ w, long long id) {
  const long long fs = g.fstride;
  const long long sd[3] = {1, g.pitch, g.plane};
  const double i12h = g.i12h;
  const double chi = w[id];
  const double alp = (double)__ldg(st + F_ALP * fs + id) + 1.0;  // stored as alpha - 1
  const double trK = (double)__ldg(st + F_TRK * fs + id);
  double beta[3], divb = 0.0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    beta[d] = (double)__ldg(st + (F_BETA + d) * fs + id);
    divb += d1u<double, float>(st + (F_BETA + d) * fs + id, sd[d]) * i12h;
  }
  double r = g.use_w ? (chi * (1.0 / 3.0)) * (alp * trK - divb)
                     : (-1.0 / 6.0) * alp * trK + divb * (1.0 / 6.0);
  const double kap = g.kos;
  const double cko[7] = {1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0};
  double bh[3];
#pragma unroll
  for (int d = 0; d < 3; d++) bh[d] = fabs(beta[d]) * i12h;
  r = fma(fma(-10.0, bh[0] + bh[1] + bh[2], -60.0 * kap), chi, r);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const bool pos = beta[d] >= 0.0;
#pragma unroll
    for (int m = -3; m <= 3; m++)
      if (m != 0) r = fma(fma(bh[d], up_coef(pos, m), kap * cko[m + 3]), w[id + m * sd[d]], r);
  }
  return r;
}

// Fused stage at interior point (ii, jj, kk), mixed precision; the accessor
// says where each field of the stage input is read from.  KS64: the k-sum of
// every field is float64 (a.ksum64; the ksum_fp64 option), a separate
// instantiation so that the default kernels keep their register allocation.
template <typename A, bool KS64 = false>
__device__ __forceinline__ void stage_point_mixed_acc(const Grid& g, const StageArgsMixed& a,
                                                      const A& acc, int ii, int jj, int kk) {
  const int i = ii + GH, j = jj + GH, k = kk + GH;
  const long long id = lin(g, i, j, k);
  const long long fs = g.fstride;
  // The combine's inputs (stages 2-3: base and k-sum; stage 4: k-sum and
  // y_n) are loaded before the right-hand side: issued after it, at 255
  // registers and 8 warps per SM, their latency was exposed (a third of the
  // step).  What the compiler cannot keep in registers it spills to local
  // memory, which comes back from L1.
  float pk[NF], ps[NF];
  double py[NF];
  constexpr bool ks64 = KS64;  // float64 k-sum of every field (ksum_fp64)
  if (a.mode == MODE_MID) {
#pragma unroll
    for (int f = 1; f < NF; f++) {
      ps[f] = a.src0[f * fs + id];
      if (!ks64) pk[f] = a.ksum[f * fs + id];
    }
  } else if (a.mode == MODE_LAST) {
#pragma unroll
    for (int f = 1; f < NF; f++) {
      if (!ks64) pk[f] = a.ksum[f * fs + id];
      py[f] = a.yn[f * fs + id];
    }
  }
  float r[NF];
  rhs_point_acc<float, float, true>(g, acc, i, j, k, r);
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
  if (a.mode == MODE_LAST) {
    // y_{n+1} = y_n + dt/6 (k1 + 2 k2 + 2 k3 + k4), the only float64 update of the step
    {
      const double v = fma(a.b_dt, a.ksumw[id] + rchi, a.yn[id]);
      a.yn[id] = v;
      a.out0[id] = (float)(v - background(g, F_CHI));
      a.out0w[id] = v;
    }
#pragma unroll
    for (int f = 1; f < NF; f++) {
      const long long o = f * fs + id;
      const double v = fma(a.b_dt, ks64 ? a.ksum64[o] + (double)r[f] : (double)(pk[f] + r[f]), py[f]);
      a.yn[o] = v;
      a.out0[o] = (float)(v - background(g, f));
    }
    return;
  }
  const float af = a.a_dtf;
  {
    const double v = fma(a.a_dt, rchi, a.src0w[id]);
    a.out0w[id] = v;
    a.out0[id] = (float)(v - background(g, F_CHI));
    a.ksumw[id] = a.mode == MODE_FIRST ? rchi : fma(2.0, rchi, a.ksumw[id]);
  }
#pragma unroll
  for (int f = 1; f < NF; f++) {
    const long long o = f * fs + id;
    a.out0[o] = fmaf(af, r[f], a.mode == MODE_FIRST ? a.src0[o] : ps[f]);
    if (ks64)
      a.ksum64[o] = a.mode == MODE_FIRST ? (double)r[f] : fma(2.0, (double)r[f], a.ksum64[o]);
    else
      a.ksum[o] = a.mode == MODE_FIRST ? r[f] : fmaf(2.0f, r[f], pk[f]);
  }
}

template <bool KS64 = false>
__device__ __forceinline__ void stage_point_mixed(const Grid& g, const StageArgsMixed& a, int ii,
                                                  int jj, int kk) {
  const GlobalAcc<float> acc(g, a.src, lin(g, ii + GH, jj + GH, kk + GH));
  stage_point_mixed_acc<GlobalAcc<float>, KS64>(g, a, acc, ii, jj, kk);
}

// ------------------------------------------------------------ double-word

// Fused stage at interior point (ii, jj, kk), double-word arithmetic.  XSEG,
// YROWS, ZS as for the float64 stage (stage_point_fp64): full 32-point rows
// share first differences across lanes for D_x D_y and D_x D_z, full blocks
// share them across rows through shared memory for D_y D_z.
template <int XSEG = 0, int YROWS = 0, int ZS = 1>
__device__ __forceinline__ void stage_point_ff(const Grid& g, const StageArgsFF& a, int ii, int jj, int kk) {
  const int i = ii + GH, j = jj + GH, k = kk + GH;
  const long long id = lin(g, i, j, k);
  ff r[NF];
  rhs_point<ff, float2, false, XSEG, YROWS, ZS>(g, a.src, id, i, j, k, r);
  const long long fs = g.fstride;
  if (a.mode == MODE_RHS) {
#pragma unroll
    for (int f = 0; f < NF; f++) a.rhs[f * fs + id] = ff_to_double(r[f]);
    return;
  }
  if (a.kshell && on_shell(g, ii, jj, kk)) {
#pragma unroll
    for (int f = 0; f < NF; f++) a.kshell[f * fs + id] = r[f].f2();
  }
  if (a.mode == MODE_LAST) {
#pragma unroll
    for (int f = 0; f < NF; f++) {
      const long long o = f * fs + id;
      const double v = fma(a.b_dt, a.ksum[o] + ff_to_double(r[f]), a.yn[o]);
      a.yn[o] = v;
      a.out0[o] = ff_from_double(v).f2();
    }
    return;
  }
  const ff adt(a.a_hi, a.a_lo);
#pragma unroll
  for (int f = 0; f < NF; f++) {
    const long long o = f * fs + id;
    a.out0[o] = ff_fma(adt, r[f], ff(__ldg(a.src0 + o))).f2();
    const double kd = ff_to_double(r[f]);
    a.ksum[o] = a.mode == MODE_FIRST ? kd : fma(2.0, kd, a.ksum[o]);
  }
}

}  // namespace bssn
