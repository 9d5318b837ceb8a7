// Per-ghost-point outer boundary work (Sommerfeld condition, periodic copy),
// shared by the single-grid kernels (k_boundary.cu) and the batched kernels
// (k_batch.cu).
#pragma once
#include "bssn_internal.cuh"
#include "rhs_point.cuh"

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

// A stored value in arithmetic C (a double-word value {hi, lo} to float64).
template <typename C, typename S>
__device__ __forceinline__ C cvt(S v) {
  return (C)v;
}
template <>
__device__ __forceinline__ double cvt<double, float2>(float2 v) {
  return (double)v.x + (double)v.y;
}
template <>
__device__ __forceinline__ ff cvt<ff, float2>(float2 v) {
  return ff(v);
}

// Radiative right-hand side of field f at stored point I in arithmetic C;
// p points at the field's value there; ns = (x / r) / (2h), the normal scaled
// by the difference weight (formed once per point for all fields), ir = 1 / r.
template <typename C, typename S, bool DEV = false>
__device__ __forceinline__ C rad_at(const Grid& g, const S* __restrict__ p, int f, const int I[3],
                                    const C ns[3], C ir) {
  const long long sd[3] = {1, g.pitch, g.plane};
  const int dims[3] = {g.sx, g.sy, g.sz};
  const bool one = (f == F_ALP || (f == F_CHI && g.use_w) || f == F_GT + 0 || f == F_GT + 3 ||
                   f == F_GT + 5);
  const C X0 = (DEV || !one) ? C(0) : C(1);  // DEV: p holds X - X0 already
  const C v0 = (f == F_ALP || f == F_TRK) ? C(1.4142135623730951) : C(1);
  C s = (cvt<C>(p[0]) - X0) * ir;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const long long q = sd[d];
    C der;
    if (I[d] >= 1 && I[d] + 1 < dims[d])
      der = cvt<C>(p[q]) - cvt<C>(p[-q]);
    else if (I[d] + 1 >= dims[d])
      der = C(3) * cvt<C>(p[0]) - C(4) * cvt<C>(p[-q]) + cvt<C>(p[-2 * q]);
    else
      der = -(C(3) * cvt<C>(p[0]) - C(4) * cvt<C>(p[q]) + cvt<C>(p[2 * q]));
    s = fmaT<C>(ns[d], der, s);
  }
  return -v0 * s;
}

// Geometry of one ghost point: its anchor and the radial factors.
struct GhostGeo {
  int I[3], A[3];
  long long ib, ia;
  double nb[3], na[3], irb, ira, fac;
  double nbs[3], nas[3];  // nb, na times 1/(2h) (rad_at)
};

__device__ __forceinline__ void ghost_geo(const Grid& g, unsigned q, GhostGeo& G) {
  ghost_decode(g, q, G.I[0], G.I[1], G.I[2]);
  const int n[3] = {g.n0, g.n1, g.n2};
  // walk to the anchor: each step moves one layer inward along the summed normal
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int a = G.I[d];
    if (a < GH) a = GH;
    else if (a >= GH + n[d]) a = GH + n[d] - 1;
    G.A[d] = a;
  }
  double xb[3], xa[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    xb[d] = coordv(g, d, G.I[d]);
    xa[d] = coordv(g, d, G.A[d]);
  }
  const double rb = sqrt(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2]);
  const double ra = sqrt(xa[0] * xa[0] + xa[1] * xa[1] + xa[2] * xa[2]);
  G.irb = 1.0 / rb;
  G.ira = 1.0 / ra;
  G.fac = (ra * G.irb) * (ra * G.irb);
#pragma unroll
  for (int d = 0; d < 3; d++) {
    G.nb[d] = xb[d] * G.irb;
    G.na[d] = xa[d] * G.ira;
    G.nbs[d] = G.nb[d] * g.i2h;
    G.nas[d] = G.na[d] * g.i2h;
  }
  G.ib = lin(g, G.I[0], G.I[1], G.I[2]);
  G.ia = lin(g, G.A[0], G.A[1], G.A[2]);
}

// Geometry table of the float64 Sommerfeld boundary, one entry per ghost
// point q (formed once per context by ghost_geo, so the same values): the
// stored indices packed in 21 bits each, and nbs[3], irb, fac.
constexpr int GEO_DOUBLES = 5;
__host__ __device__ inline size_t ghost_table_bytes(const Grid& g) {
  return (size_t)ghost_count(g) * (GEO_DOUBLES * sizeof(double) + sizeof(long long));
}
__device__ __forceinline__ void ghost_table_fill(const Grid& g, unsigned q, double* __restrict__ tab,
                                                 long long* __restrict__ itab) {
  GhostGeo G;
  ghost_geo(g, q, G);
  const size_t n = ghost_count(g);
  tab[0 * n + q] = G.nbs[0];
  tab[1 * n + q] = G.nbs[1];
  tab[2 * n + q] = G.nbs[2];
  tab[3 * n + q] = G.irb;
  tab[4 * n + q] = G.fac;
  itab[q] = (long long)G.I[0] | ((long long)G.I[1] << 21) | ((long long)G.I[2] << 42);
}

// float64 path from the table, after the anchor pass: ghost point q, fields
// [F0, F1) (a group of the 24 per thread, their loads in flight together).
template <int F0, int F1>
__device__ __forceinline__ void sommerfeld_point_fp64_tab(const Grid& g, const StageArgs& a,
                                                          const double* __restrict__ kanchor,
                                                          const double* __restrict__ tab,
                                                          const long long* __restrict__ itab, unsigned q) {
  const size_t n = ghost_count(g);
  const long long pk = itab[q];
  const int I[3] = {(int)(pk & 0x1fffff), (int)((pk >> 21) & 0x1fffff), (int)((pk >> 42) & 0x1fffff)};
  const int nn[3] = {g.n0, g.n1, g.n2};
  int A[3];
#pragma unroll
  for (int d = 0; d < 3; d++) A[d] = I[d] < GH ? GH : (I[d] >= GH + nn[d] ? GH + nn[d] - 1 : I[d]);
  const double nbs[3] = {tab[q], tab[n + q], tab[2 * n + q]};
  const double irb = tab[3 * n + q], fac = tab[4 * n + q];
  const long long ib = lin(g, I[0], I[1], I[2]), ia = lin(g, A[0], A[1], A[2]);
  const long long fs = g.fstride;
  const int nf = g.shift == BSSN_SHIFT_FROZEN ? F_BETA : NF;
#pragma unroll
  for (int f = F0; f < F1; f++) {
    double rhs = 0.0;
    if (f < nf) {
      const double radb = rad_at<double, double>(g, a.src + f * fs + ib, f, I, nbs, irb);
      rhs = fma(fac, kanchor[f * fs + ia], radb);
    }
    const long long o = f * fs + ib;
    if (a.mode == MODE_LAST) {
      a.yn[o] = fma(a.b_dt, a.ksum[o] + rhs, a.yn[o]);
    } else {
      a.out0[o] = fma(a.a_dt, rhs, a.src0[o]);
      a.ksum[o] = a.mode == MODE_FIRST ? rhs : fma(2.0, rhs, a.ksum[o]);
    }
  }
}

// float64 path, anchor pass: interior point q of the boundary shell, fields
// [F0, F1): k - rad at the anchor, in place of the k the stage kernel left in
// kanchor (the same operations the ghost points of that anchor would repeat,
// one to three layers and up to eight neighbours over; see sommerfeld_point_fp64).
template <int F0 = 0, int F1 = NF>
__device__ __forceinline__ void sommerfeld_anchor_fp64(const Grid& g, const StageArgs& a,
                                                       double* __restrict__ kanchor, unsigned q) {
  int ii, jj, kk;
  shell_decode(g, q, ii, jj, kk);
  const int A[3] = {ii + GH, jj + GH, kk + GH};
  double xa[3];
#pragma unroll
  for (int d = 0; d < 3; d++) xa[d] = coordv(g, d, A[d]);
  // as ghost_geo forms the anchor's factors
  const double ra = sqrt(xa[0] * xa[0] + xa[1] * xa[1] + xa[2] * xa[2]);
  const double ira = 1.0 / ra;
  double nas[3];
#pragma unroll
  for (int d = 0; d < 3; d++) nas[d] = (xa[d] * ira) * g.i2h;
  const long long ia = lin(g, A[0], A[1], A[2]);
  const long long fs = g.fstride;
  const int nf = g.shift == BSSN_SHIFT_FROZEN ? F_BETA : NF;
#pragma unroll
  for (int f = F0; f < F1; f++) {
    if (f >= nf) break;
    const double rada = rad_at<double, double>(g, a.src + f * fs + ia, f, A, nas, ira);
    kanchor[f * fs + ia] -= rada;
  }
}

// float64 path: ghost point q, all fields.  PRE: kanchor already holds
// k - rad at the anchor (the anchor pass ran), else k itself.
template <bool PRE = false>
__device__ __forceinline__ void sommerfeld_point_fp64(const Grid& g, const StageArgs& a,
                                                      const double* __restrict__ kanchor, unsigned q) {
  GhostGeo G;
  ghost_geo(g, q, G);
  const long long fs = g.fstride;
  const int nf = g.shift == BSSN_SHIFT_FROZEN ? F_BETA : NF;
  for (int f = 0; f < NF; f++) {
    double rhs = 0.0;
    if (f < nf) {
      const double radb = rad_at<double, double>(g, a.src + f * fs + G.ib, f, G.I, G.nbs, G.irb);
      if (PRE && a.mode != MODE_RHS) {
        rhs = fma(G.fac, kanchor[f * fs + G.ia], radb);
      } else {
        const double rada = rad_at<double, double>(g, a.src + f * fs + G.ia, f, G.A, G.nas, G.ira);
        const double ka = (a.mode == MODE_RHS) ? a.rhs[f * fs + G.ia] : kanchor[f * fs + G.ia];
        rhs = fma(G.fac, ka - rada, radb);
      }
    }
    const long long o = f * fs + G.ib;
    if (a.mode == MODE_RHS) {
      a.rhs[o] = rhs;
    } else if (a.mode == MODE_LAST) {
      a.yn[o] = fma(a.b_dt, a.ksum[o] + rhs, a.yn[o]);
    } else {
      a.out0[o] = fma(a.a_dt, rhs, a.src0[o]);
      a.ksum[o] = a.mode == MODE_FIRST ? rhs : fma(2.0, rhs, a.ksum[o]);
    }
  }
}

// mixed path: ghost point q, field f; float arithmetic, W in float64; RK4
// roles as in the stage kernel.
__device__ __forceinline__ void sommerfeld_point_mixed(const Grid& g, const StageArgsMixed& a,
                                                       const float* __restrict__ kanchor, unsigned q,
                                                       int f) {
  const long long fs = g.fstride;
  const int nf = g.shift == BSSN_SHIFT_FROZEN ? F_BETA : NF;
  int I[3], A[3];
  ghost_decode(g, q, I[0], I[1], I[2]);
  const int n[3] = {g.n0, g.n1, g.n2};
#pragma unroll
  for (int d = 0; d < 3; d++) A[d] = I[d] < GH ? GH : (I[d] >= GH + n[d] ? GH + n[d] - 1 : I[d]);
  const long long ib = lin(g, I[0], I[1], I[2]);
  const long long ia = lin(g, A[0], A[1], A[2]);
  const long long o = f * fs + ib;
  if (f == F_CHI) {
    GhostGeo G;
    ghost_geo(g, q, G);
    const double radb = rad_at<double, double>(g, a.srcw + ib, f, I, G.nbs, G.irb);
    const double rada = rad_at<double, double>(g, a.srcw + ia, f, A, G.nas, G.ira);
    const double ka = (a.mode == MODE_RHS) ? a.rhs[ia] : (double)kanchor[ia];
    const double rhs = fma(G.fac, ka - rada, radb);
    if (a.mode == MODE_RHS) {
      a.rhs[o] = rhs;
    } else if (a.mode == MODE_LAST) {
      const double v = fma(a.b_dt, a.ksumw[ib] + rhs, a.yn[ib]);
      a.yn[ib] = v;
      a.out0[ib] = (float)(v - background(g, F_CHI));
      a.out0w[ib] = v;
    } else {
      const double v = fma(a.a_dt, rhs, a.src0w[ib]);
      a.out0w[ib] = v;
      a.out0[ib] = (float)(v - background(g, F_CHI));
      a.ksumw[ib] = a.mode == MODE_FIRST ? rhs : fma(2.0, rhs, a.ksumw[ib]);
    }
    return;
  }
  float rhs = 0.0f;
  if (f < nf) {
    float xb[3], xa[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      xb[d] = fmaf((float)(I[d] - GH) + 0.5f, g.hf, g.xminf[d]);
      xa[d] = fmaf((float)(A[d] - GH) + 0.5f, g.hf, g.xminf[d]);
    }
    const float irb = rsqrtf(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2]);
    const float ira = rsqrtf(xa[0] * xa[0] + xa[1] * xa[1] + xa[2] * xa[2]);
    const float nbs[3] = {xb[0] * irb * g.i2hf, xb[1] * irb * g.i2hf, xb[2] * irb * g.i2hf};
    const float nas[3] = {xa[0] * ira * g.i2hf, xa[1] * ira * g.i2hf, xa[2] * ira * g.i2hf};
    const float fac = (irb / ira) * (irb / ira);
    const float radb = rad_at<float, float, true>(g, a.src + o, f, I, nbs, irb);
    const float rada = rad_at<float, float, true>(g, a.src + f * fs + ia, f, A, nas, ira);
    const float ka = (a.mode == MODE_RHS) ? (float)a.rhs[f * fs + ia] : kanchor[f * fs + ia];
    rhs = fmaf(fac, ka - rada, radb);
  }
  if (a.mode == MODE_RHS) {
    a.rhs[o] = (double)rhs;
  } else if (a.mode == MODE_LAST) {
    const double ks = a.ksum64 ? a.ksum64[o] + (double)rhs : (double)(a.ksum[o] + rhs);
    const double v = fma(a.b_dt, ks, a.yn[o]);
    a.yn[o] = v;
    a.out0[o] = (float)(v - background(g, f));
  } else {
    a.out0[o] = fmaf(a.a_dtf, rhs, a.src0[o]);
    if (a.ksum64)
      a.ksum64[o] = a.mode == MODE_FIRST ? (double)rhs : fma(2.0, (double)rhs, a.ksum64[o]);
    else
      a.ksum[o] = a.mode == MODE_FIRST ? rhs : fmaf(2.0f, rhs, a.ksum[o]);
  }
}

// mixed path, ghost point q, fields [F0, F1): the same per-field arithmetic
// as sommerfeld_point_mixed with the geometry (index decode, anchor,
// coordinates, normals) formed once for the group's float fields; W (field 0,
// when in the group) in float64.  UNROLL: the field loop unrolled, so that the
// group's loads are in flight together.
template <int F0, int F1, bool UNROLL>
__device__ __forceinline__ void sommerfeld_point_mixed_fields(const Grid& g, const StageArgsMixed& a,
                                                              const float* __restrict__ kanchor, unsigned q) {
  if constexpr (F0 == 0) sommerfeld_point_mixed(g, a, kanchor, q, F_CHI);  // W: float64 geometry and arithmetic
  constexpr int FB = F0 == 0 ? 1 : F0;
  const long long fs = g.fstride;
  const int nf = g.shift == BSSN_SHIFT_FROZEN ? F_BETA : NF;
  int I[3], A[3];
  ghost_decode(g, q, I[0], I[1], I[2]);
  const int n[3] = {g.n0, g.n1, g.n2};
#pragma unroll
  for (int d = 0; d < 3; d++) A[d] = I[d] < GH ? GH : (I[d] >= GH + n[d] ? GH + n[d] - 1 : I[d]);
  const long long ib = lin(g, I[0], I[1], I[2]);
  const long long ia = lin(g, A[0], A[1], A[2]);
  float xb[3], xa[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    xb[d] = fmaf((float)(I[d] - GH) + 0.5f, g.hf, g.xminf[d]);
    xa[d] = fmaf((float)(A[d] - GH) + 0.5f, g.hf, g.xminf[d]);
  }
  const float irb = rsqrtf(xb[0] * xb[0] + xb[1] * xb[1] + xb[2] * xb[2]);
  const float ira = rsqrtf(xa[0] * xa[0] + xa[1] * xa[1] + xa[2] * xa[2]);
  // normals times 1/(2h) (rad_at)
  const float nbs[3] = {xb[0] * irb * g.i2hf, xb[1] * irb * g.i2hf, xb[2] * irb * g.i2hf};
  const float nas[3] = {xa[0] * ira * g.i2hf, xa[1] * ira * g.i2hf, xa[2] * ira * g.i2hf};
  const float fac = (irb / ira) * (irb / ira);
#pragma unroll (UNROLL ? F1 - FB : 1)
  for (int f = FB; f < F1; f++) {
    const long long o = f * fs + ib;
    float rhs = 0.0f;
    if (f < nf) {
      const float radb = rad_at<float, float, true>(g, a.src + o, f, I, nbs, irb);
      const float rada = rad_at<float, float, true>(g, a.src + f * fs + ia, f, A, nas, ira);
      const float ka = (a.mode == MODE_RHS) ? (float)a.rhs[f * fs + ia] : kanchor[f * fs + ia];
      rhs = fmaf(fac, ka - rada, radb);
    }
    if (a.mode == MODE_RHS) {
      a.rhs[o] = (double)rhs;
    } else if (a.mode == MODE_LAST) {
      const double ks = a.ksum64 ? a.ksum64[o] + (double)rhs : (double)(a.ksum[o] + rhs);
      const double v = fma(a.b_dt, ks, a.yn[o]);
      a.yn[o] = v;
      a.out0[o] = (float)(v - background(g, f));
    } else {
      a.out0[o] = fmaf(a.a_dtf, rhs, a.src0[o]);
      if (a.ksum64)
        a.ksum64[o] = a.mode == MODE_FIRST ? (double)rhs : fma(2.0, (double)rhs, a.ksum64[o]);
      else
        a.ksum[o] = a.mode == MODE_FIRST ? rhs : fmaf(2.0f, rhs, a.ksum[o]);
    }
  }
}

// every field in one thread (the batched boundary kernel)
__device__ __forceinline__ void sommerfeld_point_mixed_all(const Grid& g, const StageArgsMixed& a,
                                                           const float* __restrict__ kanchor, unsigned q) {
  sommerfeld_point_mixed_fields<0, NF, false>(g, a, kanchor, q);
}

// Periodic ghosts: copy from the wrapped interior point, all fields (and the
// float64 W array of a mixed stage buffer when w is non-null).
template <typename S>
__device__ __forceinline__ void periodic_point(const Grid& g, S* __restrict__ y,
                                               double* __restrict__ w, unsigned q) {
  int i, j, k;
  ghost_decode(g, q, i, j, k);
  const int si = GH + ((i - GH) % g.n0 + g.n0) % g.n0;
  const int sj = GH + ((j - GH) % g.n1 + g.n1) % g.n1;
  const int sk = GH + ((k - GH) % g.n2 + g.n2) % g.n2;
  const long long d = lin(g, i, j, k), s = lin(g, si, sj, sk);
  for (int f = 0; f < NF; f++) y[f * g.fstride + d] = y[f * g.fstride + s];
  if (w) w[d] = w[s];
}

// Sommerfeld boundary of the double-word path: ghost point q, all fields (the
// closed form of the layered recursion, as on the float64 path).  The
// geometry is formed once per point in float64 and rounded to double-word
// values; the radiative terms run in double-word arithmetic on the stage
// values; the k-sum and y_n as in the stage kernel.
__device__ __forceinline__ void sommerfeld_point_ff(const Grid& g, const StageArgsFF& a,
                                                    const float2* __restrict__ kanchor, unsigned q) {
  GhostGeo G;
  ghost_geo(g, q, G);
  ff nbs[3], nas[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    nbs[d] = ff_from_double(G.nbs[d]);
    nas[d] = ff_from_double(G.nas[d]);
  }
  const ff irb = ff_from_double(G.irb), ira = ff_from_double(G.ira), fac = ff_from_double(G.fac);
  const ff adt(a.a_hi, a.a_lo);
  const long long fs = g.fstride;
  const int nf = g.shift == BSSN_SHIFT_FROZEN ? F_BETA : NF;
  for (int f = 0; f < NF; f++) {
    ff rhs(0.0f, 0.0f);
    if (f < nf) {
      const ff radb = rad_at<ff, float2>(g, a.src + f * fs + G.ib, f, G.I, nbs, irb);
      const ff rada = rad_at<ff, float2>(g, a.src + f * fs + G.ia, f, G.A, nas, ira);
      const ff ka = (a.mode == MODE_RHS) ? ff_from_double(a.rhs[f * fs + G.ia]) : ff(kanchor[f * fs + G.ia]);
      rhs = ff_fma(fac, ka - rada, radb);
    }
    const long long o = f * fs + G.ib;
    if (a.mode == MODE_RHS) {
      a.rhs[o] = ff_to_double(rhs);
    } else if (a.mode == MODE_LAST) {
      const double v = fma(a.b_dt, a.ksum[o] + ff_to_double(rhs), a.yn[o]);
      a.yn[o] = v;
      a.out0[o] = ff_from_double(v).f2();
    } else {
      a.out0[o] = ff_fma(adt, rhs, ff(a.src0[o])).f2();
      const double kd = ff_to_double(rhs);
      a.ksum[o] = a.mode == MODE_FIRST ? kd : fma(2.0, kd, a.ksum[o]);
    }
  }
}

}  // namespace bssn
