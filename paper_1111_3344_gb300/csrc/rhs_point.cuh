// Pointwise BSSN right-hand side on the device (arXiv:1111.3344, Sec.
// "Spacetime Curvature Evolution": evolution equations for alpha, K, beta, B,
// phi, gt, At, Gt with m = 1 in vacuum; Ricci pieces Rt_ij and Rphi_ij; 1+log
// / harmonic / geodesic slicing; Gamma-driver shift with q(r)).
//
// Formulation (same discrete operator as the statement in the paper; the
// arrangement is chosen to cut float64 instructions, the binding resource on
// GB300):
//  - symmetric tensors held as 6 components; gt^{ij} by cofactors over det;
//  - second derivatives are consumed as they are produced (the
//    gt^{kl} d_k d_l contractions are accumulated pair by pair) to keep the
//    live set small;
//  - d_l gt^{lk} = -gt^{la} gt^{kb} d_l gt_ab from the metric stencils, in Rt
//    and the Gt equation; only gt_k(i d_j) Gt^k uses the evolved Gt;
//  - W variant: d phi = -d W / (2W), d d phi = -dd W / (2W) + 2 dphi dphi,
//    e^{-4 phi} = W^2 (W floored where it divides);
//  - advection beta^j d_j X with the lopsided stencil on the upwind side,
//    written as |beta^j| times the mirrored stencil; KO as
//    +eps/(64h) sum_d delta_d^6 X.
#pragma once
#include "bssn_internal.cuh"

namespace bssn {

template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c);
template <>
__device__ __forceinline__ double fmaT<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmaT<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ ff fmaT<ff>(ff a, ff b, ff c) { return ff_fma(a, b, c); }

// |x| and e^x in the arithmetic type
template <typename T>
__device__ __forceinline__ T absT(T x) { return fabs(x); }
template <>
__device__ __forceinline__ ff absT<ff>(ff x) { return ff_fabs(x); }
template <typename T>
__device__ __forceinline__ T expT(T x) { return exp(x); }
template <>
__device__ __forceinline__ ff expT<ff>(ff x) { return ff_exp(x); }

template <typename T, typename S>
__device__ __forceinline__ T ldg(const S* p) {
  return T(__ldg(p));
}

// Field access of rhs_point.  An accessor gives, for field f at the point,
// a pointer, the strides of the three axes and a load; the compiler resolves
// the field-dependent choices because f is a constant after unrolling.
// GlobalAcc: every field read from the global register (read-only path).
template <typename S>
struct GlobalAcc {
  const S* __restrict__ st;
  long long id, fs, sd[3];
  __device__ __forceinline__ GlobalAcc(const Grid& g, const S* __restrict__ st_, long long id_)
      : st(st_), id(id_), fs(g.fstride), sd{1, g.pitch, g.plane} {}
  __device__ __forceinline__ const S* ptr(int f) const { return st + (long long)f * fs + id; }
  __device__ __forceinline__ long long s(int, int d) const { return sd[d]; }
  template <typename T>
  __device__ __forceinline__ T ld(int, const S* p) const { return T(__ldg(p)); }
};

// Accessors whose derivatives and advection/dissipation sums were computed
// beforehand (the split mixed stage, k_stage_split.cu) say so here; the
// right-hand side then adds acc.advko(f) instead of applying the 7-point
// stencils itself.
template <typename A>
struct is_precomputed {
  static constexpr bool value = false;
};

// 8 (f1 - f-1) - (f2 - f-2): 12 h times the 4th-order first derivative.
template <typename T, typename A, typename P>
__device__ __forceinline__ T d1u(const A& acc, int f, const P* p, long long s) {
  T a = acc.template ld<T>(f, p + s) - acc.template ld<T>(f, p - s);
  T b = acc.template ld<T>(f, p + 2 * s) - acc.template ld<T>(f, p - 2 * s);
  return fmaT<T>(T(8), a, -b);
}
// 16 (f1 + f-1) - (f2 + f-2) - 30 f0: 12 h^2 times the 4th-order second derivative.
// In float the same sum is formed from differences to the centre value,
// 16 ((f1 - f0) + (f-1 - f0)) - ((f2 - f0) + (f-2 - f0)): neighbour differences
// are (nearly) exact, so the rounding scales with h f' instead of |f| (the
// plain form loses |f| / (h^2 f'') of float's 24 bits).  Float64 keeps the
// cheaper plain form.
template <typename T, typename A, typename P>
__device__ __forceinline__ T d2u(const A& acc, int f, const P* p, long long s, T f0) {
  if constexpr (is_f32<T>) {
    T a = (acc.template ld<T>(f, p + s) - f0) + (acc.template ld<T>(f, p - s) - f0);
    T b = (acc.template ld<T>(f, p + 2 * s) - f0) + (acc.template ld<T>(f, p - 2 * s) - f0);
    return fmaT<T>(T(16), a, -b);
  } else {
    T a = acc.template ld<T>(f, p + s) + acc.template ld<T>(f, p - s);
    T b = acc.template ld<T>(f, p + 2 * s) + acc.template ld<T>(f, p - 2 * s);
    return fmaT<T>(T(-30), f0, fmaT<T>(T(16), a, -b));
  }
}
// D1_a D1_b (a != b): 144 h^2 times the mixed derivative.
template <typename T, typename A, typename P>
__device__ __forceinline__ T dmu(const A& acc, int f, const P* p, long long sa, long long sb) {
  T a = d1u<T>(acc, f, p + sa, sb) - d1u<T>(acc, f, p - sa, sb);
  T b = d1u<T>(acc, f, p + 2 * sa, sb) - d1u<T>(acc, f, p - 2 * sa, sb);
  return fmaT<T>(T(8), a, -b);
}
// D1_x D1_b of field f (b = y or z) for a warp whose 32 lanes hold 32
// consecutive x points of one row: v is this point's first difference along b
// (already formed, scaled by 1/(12h)); the lanes x-1, x+1, x-2, x+2 hold
// theirs, so only the two lanes at each end of the row form one more
// (at x -+ 2), and the mixed difference costs 3 float64 operations instead
// of 15.  Same stencil as dmu (D1 along x applied to D1 along b); the result
// is 12 h times the mixed derivative (v already carries 1/(12h)).
__device__ __forceinline__ double shflT(double v, int src, int W) { return __shfl_sync(0xffffffffu, v, src, W); }
__device__ __forceinline__ ff shflT(ff v, int src, int W) {
  return ff(__shfl_sync(0xffffffffu, v.hi, src, W), __shfl_sync(0xffffffffu, v.lo, src, W));
}
template <int W, typename T, typename A, typename P>
__device__ __forceinline__ T dmx_shfl(const A& acc, int f, const P* p, long long sb, T v, T i12h) {
  const int lane = threadIdx.x & (W - 1);
  const bool lo = lane < 2, hi = lane >= W - 2;
  T ve = T(0);
  if (lo || hi) ve = d1u<T>(acc, f, p + (lo ? -2 : 2), sb) * i12h;  // x - 2 or x + 2
  const T sm2 = shflT(v, lane - 2, W);
  const T sm1 = shflT(v, lane - 1, W);
  const T sp1 = shflT(v, lane + 1, W);
  const T sp2 = shflT(v, lane + 2, W);
  const T e1 = shflT(ve, 1, W);       // lane 1 holds x_0 - 1
  const T ew = shflT(ve, W - 2, W);   // lane W-2 holds x_{W-1} + 1
  const T vm2 = lane >= 2 ? sm2 : ve;
  const T vm1 = lane >= 1 ? sm1 : e1;
  const T vp1 = lane <= W - 2 ? sp1 : ew;
  const T vp2 = lane <= W - 3 ? sp2 : ve;
  return fmaT<T>(T(8), vp1 - vm1, -(vp2 - vm2));
}
// The same mixed difference with the four first differences past the ends of
// the row already formed (float64 full blocks): xe[0..3] hold them at
// x_0 - 2, x_0 - 1, x_{W-1} + 1, x_{W-1} + 2, in shared memory.
template <int W, typename T>
__device__ __forceinline__ T dmx_pre(T v, const T* xe) {
  const int lane = threadIdx.x & (W - 1);
  const T sm2 = shflT(v, lane - 2, W);
  const T sm1 = shflT(v, lane - 1, W);
  const T sp1 = shflT(v, lane + 1, W);
  const T sp2 = shflT(v, lane + 2, W);
  // indices clamped to 0..3 on every lane, so that no lane reads past xe
  const T vm2 = lane >= 2 ? sm2 : xe[lane < 2 ? lane : 0];
  const T vm1 = lane >= 1 ? sm1 : xe[1];
  const T vp1 = lane <= W - 2 ? sp1 : xe[2];
  const T vp2 = lane <= W - 3 ? sp2 : xe[lane >= W - 2 ? lane - W + 4 : 3];
  return fmaT<T>(T(8), vp1 - vm1, -(vp2 - vm2));
}

// x-mixed difference of the q-th of the 11 twice-differenced fields (gt_ij,
// phi|W, alpha, beta^i) along axis b (1 or 2): from the staged end-of-row
// values on float64 full blocks, else with the end lanes forming their own.
// (Double-word blocks keep the end lanes' own: the 88 values per warp cost
// them shared memory that their register spills use as L1, and the stage
// measured 3 % slower, 30 % in the batch.)
template <int W, int YROWS, typename T, typename A, typename P>
__device__ __forceinline__ T dmx_row(const A& acc, int f, const P* p, long long sb, T v, T i12h, const T* xep,
                                     int b, int q) {
  if constexpr (YROWS > 0 && is_f64<T>) return dmx_pre<W>(v, xep + ((b == 2 ? 11 : 0) + q) * 4);
  else return dmx_shfl<W>(acc, f, p, sb, v, i12h);
}

// Dynamic shared memory of a float64 or double-word full-block stage (32 x ty
// x tz points; 8-byte values): the first differences along z of 11 fields
// over the block's rows and two halo rows on each side, then, for float64
// (ends), per warp the 88 first differences along y and z past the ends of
// its row (dmx_pre).
static_assert(sizeof(ff) == sizeof(double), "double-word values take 8-byte slots");
__host__ __device__ constexpr size_t rows_block_smem(int ty, int tz, bool ends) {
  return ((size_t)11 * (ty + 4) * tz * 32 + (ends ? (size_t)ty * tz * 88 : 0)) * sizeof(double);
}

// the same helpers over the plain read-only global path (one field)
template <typename T, typename S>
struct PlainAcc {
  template <typename U>
  __device__ __forceinline__ U ld(int, const S* p) const { return U(__ldg(p)); }
};
template <typename T, typename S>
__device__ __forceinline__ T d1u(const S* p, long long s) {
  return d1u<T>(PlainAcc<T, S>{}, 0, p, s);
}

// Advection plus dissipation of every field as one 7-point stencil per axis.
// Along axis d the upwinded advection beta^d d_d X (lopsided stencil on the
// side the sign of beta^d selects) and the KO term eps/(64h) delta_d^6 X are
// both linear in the values X(m s_d), m = -3..3, so their sum is
//   sum_m w_d[m] X(m s_d),  w_d[m] = eps/(64h) c_KO[m] + |beta^d|/(12h) u_d[m]
// with u_d = (0, 0, -3, -10, 18, -6, 1) for beta^d >= 0 and its mirror
// (1, -6, 18, -10, -3, 0, 0) otherwise.  The weights are formed once per
// point and shared by all fields; the centre weights of the three axes are
// merged.
__device__ __forceinline__ double up_coef(bool pos, int m) {
  // u_d[m] for m in -3..3
  const double cp[7] = {0.0, 0.0, -3.0, -10.0, 18.0, -6.0, 1.0};
  const double cn[7] = {1.0, -6.0, 18.0, -10.0, -3.0, 0.0, 0.0};
  return pos ? cp[m + 3] : cn[m + 3];
}
// the same weight in the arithmetic type T (float and double-word: from the
// float constants, which hold these small integers exactly)
template <typename T>
__device__ __forceinline__ T up_coefT(bool pos, int m) {
  if constexpr (is_f64<T>) {
    return up_coef(pos, m);
  } else {
    const float cp[7] = {0.0f, 0.0f, -3.0f, -10.0f, 18.0f, -6.0f, 1.0f};
    const float cn[7] = {1.0f, -6.0f, 18.0f, -10.0f, -3.0f, 0.0f, 0.0f};
    return T(pos ? cp[m + 3] : cn[m + 3]);
  }
}

// Background value X0 of field f (1 for W, the diagonal of gt and alpha; 0
// otherwise).  The float stage buffers of the mixed path hold X - X0, so that
// float precision goes to the deviation; every stencil's weights sum to zero,
// so derivatives of the deviation are the derivatives of X.
__host__ __device__ __forceinline__ double background(const Grid& g, int f) {
  return ((f == F_CHI && g.use_w) || f == F_GT + 0 || f == F_GT + 3 || f == F_GT + 5 || f == F_ALP)
             ? 1.0 : 0.0;
}

// Right-hand side of all 24 fields at interior point (i, j, k) with linear
// index id, reading the state register st (field stride g.fstride).  DEV: the
// register holds X - X0 (mixed-path float buffers) instead of X.
// XSEG = 32: the calling warp is one full x-row of 32 points (float64 only);
// the mixed second differences involving x then share first differences
// across lanes (dmx_shfl).  XSEG = 0: every stencil evaluated by the thread.
// YROWS > 0 (with XSEG = 32): the block is 32 x YROWS x ZS points, every
// thread inside the grid, and D_y D_z takes the neighbouring rows' first
// differences along z from shared memory (11 fields x (YROWS + 4) rows x ZS x
// 32 doubles of dynamic shared memory; one barrier).
template <typename T, typename S, bool DEV, typename A, int XSEG = 0, int YROWS = 0, int ZS = 1>
__device__ __forceinline__ void rhs_point_acc(const Grid& g, const A& acc, int i, int j, int k,
                                              T out[NF]) {
  // ROLL (double-word arithmetic): a double-word operation is 7 to 15 float
  // instructions, so the fully unrolled right-hand side would be some 30,000
  // instructions of straight-line code per point, far beyond the instruction
  // cache (ncu: warps stalled mostly on instruction fetch).  The second
  // derivatives (six pairs) and the advection / dissipation stencils (24
  // fields) then run as loops over the pairs and the fields, in the same order
  // and with the same arithmetic, with their per-iteration values kept in
  // arrays indexed at run time.
  constexpr bool ROLL = std::is_same<T, ff>::value;
  const T i12h = gc<T>(g.i12h, g.i12hf, g.i12hl);
  const T i12h2 = gc<T>(g.i12h2, g.i12h2f, g.i12h2l);
  const T i144h2 = gc<T>(g.i144h2, g.i144h2f, g.i144h2l);
#define PF(f) acc.ptr(f)
#define SD(f, d) acc.s((f), (d))
#define LD(f, p) acc.template ld<T>((f), (p))

  // ---- point values (raw: as stored; chi, gt, alp: the field values)
  const T chi_r = LD(F_CHI, PF(F_CHI));
  T gt_r[6], gt[6], At[6];
#pragma unroll
  for (int m = 0; m < 6; m++) {
    gt_r[m] = LD(F_GT + m, PF(F_GT + m));
    At[m] = LD(F_AT + m, PF(F_AT + m));
  }
  T trK = LD(F_TRK, PF(F_TRK));
  const T alp_r = LD(F_ALP, PF(F_ALP));
  const T chi = DEV && g.use_w ? chi_r + T(1) : chi_r;
  const T alp = DEV ? alp_r + T(1) : alp_r;
#pragma unroll
  for (int m = 0; m < 6; m++) gt[m] = (DEV && (m == 0 || m == 3 || m == 5)) ? gt_r[m] + T(1) : gt_r[m];
  T beta[3], Bv[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    beta[a] = LD(F_BETA + a, PF(F_BETA + a));
    Bv[a] = LD(F_B + a, PF(F_B + a));
  }

  // ---- inverse conformal metric (cofactors / det); in the W variant one
  // division gives both 1/det and 1/(2W) (W floored where it divides)
  T gu[6], ihW = T(0);
  {
    T c00 = gt[3] * gt[5] - gt[4] * gt[4];
    T c01 = gt[2] * gt[4] - gt[1] * gt[5];
    T c02 = gt[1] * gt[4] - gt[2] * gt[3];
    T det = gt[0] * c00 + gt[1] * c01 + gt[2] * c02;
    T idet;
    if (g.use_w) {
      const T wf = gc<T>(g.w_floor, g.w_floorf, g.w_floorl);
      const T Wd = chi > wf ? chi : wf;
      const T r = T(1) / (det * Wd);
      idet = Wd * r;
      ihW = T(0.5) * det * r;
    } else {
      idet = T(1) / det;
    }
    gu[0] = c00 * idet;
    gu[1] = c01 * idet;
    gu[2] = c02 * idet;
    gu[3] = (gt[0] * gt[5] - gt[2] * gt[2]) * idet;
    gu[4] = (gt[1] * gt[2] - gt[0] * gt[4]) * idet;
    gu[5] = (gt[0] * gt[3] - gt[1] * gt[1]) * idet;
  }

  // ---- first derivatives
  T dgt[3][6], dchi[3], dalp[3], dK[3], db[3][3], dG[3][3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
#pragma unroll
    for (int m = 0; m < 6; m++) dgt[d][m] = d1u<T>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, d)) * i12h;
    dchi[d] = d1u<T>(acc, F_CHI, PF(F_CHI), SD(F_CHI, d)) * i12h;
    dalp[d] = d1u<T>(acc, F_ALP, PF(F_ALP), SD(F_ALP, d)) * i12h;
    dK[d] = d1u<T>(acc, F_TRK, PF(F_TRK), SD(F_TRK, d)) * i12h;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      db[d][a] = d1u<T>(acc, F_BETA + a, PF(F_BETA + a), SD(F_BETA + a, d)) * i12h;
      dG[d][a] = d1u<T>(acc, F_GAM + a, PF(F_GAM + a), SD(F_GAM + a, d)) * i12h;
    }
  }

  // ---- D_y D_z through shared memory (full blocks of full rows)
  [[maybe_unused]] T dyz[11];  // gt_ij (6), phi|W, alpha, beta^i (3)
  [[maybe_unused]] const T* xep = nullptr;  // this warp's 88 end-of-row first differences (float64)
  if constexpr (YROWS > 0 && XSEG == 32 && !is_f32<T>) {
    extern __shared__ double yz_smem[];  // 8-byte slots: float64 or double-word values
    T* yz = reinterpret_cast<T*>(yz_smem);
    constexpr int ROWS = YROWS + 4;
    const int ty = threadIdx.y, tz = threadIdx.z, lane = threadIdx.x;
    auto at = [&](int q, int row) -> T& { return yz[((q * ROWS + row) * ZS + tz) * 32 + lane]; };
    auto dz_of = [&](int q) -> T {
      return q < 6 ? dgt[2][q] : (q == 6 ? dchi[2] : (q == 7 ? dalp[2] : db[2][q - 8]));
    };
    auto field_of = [](int q) { return q < 6 ? F_GT + q : (q == 6 ? F_CHI : (q == 7 ? F_ALP : F_BETA + (q - 8))); };
    const long long sy = SD(F_CHI, 1), sz = SD(F_CHI, 2);
#pragma unroll
    for (int q = 0; q < 11; q++) at(q, ty + 2) = dz_of(q);
    if (ty < 2) {  // rows y0-2, y0-1 below the block
#pragma unroll
      for (int q = 0; q < 11; q++) at(q, ty) = d1u<T>(acc, field_of(q), PF(field_of(q)) - 2 * sy, sz) * i12h;
    }
    if (ty >= YROWS - 2) {  // rows y0+YROWS, y0+YROWS+1 above it
#pragma unroll
      for (int q = 0; q < 11; q++) at(q, ty + 4) = d1u<T>(acc, field_of(q), PF(field_of(q)) + 2 * sy, sz) * i12h;
    }
    if constexpr (is_f64<T>) {
      // The x-mixed differences need, for each of the 11 fields and for y
      // and z, the first differences at the four points past the ends of
      // this warp's row: 88 values.  All 32 lanes form them, three rounds of
      // one value each, into shared memory (item 4 p + e: pair p = field
      // q + 11 (0 for y, 1 for z), point e = x_0 - 2, x_0 - 1, x_0 + 32,
      // x_0 + 33), rather than the two lanes at each end of the row with the
      // other 30 lanes of every such instruction idle.  Same arithmetic.
      T* xe = yz + 11 * ROWS * ZS * 32 + (tz * YROWS + ty) * 88;
#pragma unroll
      for (int r = 0; r < 3; r++) {
        const int idx = r * 32 + lane;
        if (idx < 88) {
          const int pr = idx >> 2, e = idx & 3;
          const int q = pr < 11 ? pr : pr - 11;
          const int f = field_of(q);
          const int dx = (e < 2 ? e - 2 : 30 + e) - lane;  // x offset from this lane's point (unit stride)
          xe[idx] = d1u<T>(acc, f, PF(f) + dx, pr < 11 ? sy : sz) * i12h;
        }
      }
      xep = xe;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 11; q++)
      dyz[q] = fmaT<T>(T(8), at(q, ty + 3) - at(q, ty + 1), -(at(q, ty + 4) - at(q, ty)));  // x 1/(12h)
  }

  // ---- second derivatives, consumed pair by pair.  Each is formed unscaled
  // (12 h^2, 12 h or 144 h^2 times the derivative, by stencil) and its scale
  // sc goes into the weight of the contraction that takes it.
  T Rdd[6];      // -1/2 gt^{kl} d_k d_l gt_ij
  T lapb[3];     // gt^{kl} d_k d_l beta^i
  T gdiv[3];     // d_j d_k beta^k
  T ddchi[6];    // d_a d_b (phi|W)
  T ddalp[6];    // d_a d_b alpha, unscaled; times sc2[pq]
  T sc2[6];
  T g2u[6];      // gt^{ab} with the off-diagonal entries doubled (symmetric contractions)
#pragma unroll
  for (int m = 0; m < 6; m++) g2u[m] = (m == 0 || m == 3 || m == 5) ? gu[m] : T(2) * gu[m];
#pragma unroll
  for (int m = 0; m < 6; m++) Rdd[m] = T(0);
#pragma unroll
  for (int a = 0; a < 3; a++) lapb[a] = gdiv[a] = T(0);
  if constexpr (ROLL) {
    // The six pairs (a, b) as a loop that is not unrolled: the same stencils
    // and the same contractions in the same order, with the pair's strides,
    // scale and first differences picked at run time -- one copy of the code
    // instead of six (see ROLL).
    const long long s3[3] = {SD(F_GT, 0), SD(F_GT, 1), SD(F_GT, 2)};
#pragma unroll 1
    for (int pq = 0; pq < 6; pq++) {
      const int pa = pq < 3 ? 0 : (pq < 5 ? 1 : 2);
      const int pb = pq < 3 ? pq : (pq < 5 ? pq - 2 : 2);
      const long long sa = pa == 0 ? s3[0] : (pa == 1 ? s3[1] : s3[2]);
      const long long sb = pb == 0 ? s3[0] : (pb == 1 ? s3[1] : s3[2]);
      T dd[6], vb[3], vchi, valp, sc;
      if (pa == pb) {
        sc = i12h2;
#pragma unroll
        for (int m = 0; m < 6; m++) dd[m] = d2u<T>(acc, F_GT + m, PF(F_GT + m), sa, gt_r[m]);
        vchi = d2u<T>(acc, F_CHI, PF(F_CHI), sa, chi_r) * i12h2;
        valp = d2u<T>(acc, F_ALP, PF(F_ALP), sa, alp_r);
#pragma unroll
        for (int a = 0; a < 3; a++) vb[a] = d2u<T>(acc, F_BETA + a, PF(F_BETA + a), sa, beta[a]);
      } else if (XSEG > 0 && pa == 0) {
        if constexpr (XSEG > 0) {
          sc = i12h;
          const bool y = pb == 1;
#pragma unroll
          for (int m = 0; m < 6; m++)
            dd[m] = dmx_row<XSEG, YROWS>(acc, F_GT + m, PF(F_GT + m), sb, y ? dgt[1][m] : dgt[2][m], i12h, xep, pb, m);
          vchi = dmx_row<XSEG, YROWS>(acc, F_CHI, PF(F_CHI), sb, y ? dchi[1] : dchi[2], i12h, xep, pb, 6) * i12h;
          valp = dmx_row<XSEG, YROWS>(acc, F_ALP, PF(F_ALP), sb, y ? dalp[1] : dalp[2], i12h, xep, pb, 7);
#pragma unroll
          for (int a = 0; a < 3; a++)
            vb[a] = dmx_row<XSEG, YROWS>(acc, F_BETA + a, PF(F_BETA + a), sb, y ? db[1][a] : db[2][a], i12h, xep,
                                         pb, 8 + a);
        }
      } else if (YROWS > 0 && pa == 1) {  // (1, 2) from the rows' differences along z
        sc = i12h;
#pragma unroll
        for (int m = 0; m < 6; m++) dd[m] = dyz[m];
        vchi = dyz[6] * i12h;
        valp = dyz[7];
#pragma unroll
        for (int a = 0; a < 3; a++) vb[a] = dyz[8 + a];
      } else {
        sc = i144h2;
#pragma unroll
        for (int m = 0; m < 6; m++) dd[m] = dmu<T>(acc, F_GT + m, PF(F_GT + m), sa, sb);
        vchi = dmu<T>(acc, F_CHI, PF(F_CHI), sa, sb) * i144h2;
        valp = dmu<T>(acc, F_ALP, PF(F_ALP), sa, sb);
#pragma unroll
        for (int a = 0; a < 3; a++) vb[a] = dmu<T>(acc, F_BETA + a, PF(F_BETA + a), sa, sb);
      }
      ddchi[pq] = vchi;
      ddalp[pq] = valp;
      sc2[pq] = sc;
      T g2 = g2u[0];
#pragma unroll
      for (int m = 1; m < 6; m++) g2 = pq == m ? g2u[m] : g2;
      const T wb = sc * g2;
      const T w = T(-0.5) * wb;
#pragma unroll
      for (int m = 0; m < 6; m++) Rdd[m] = fmaT<T>(w, dd[m], Rdd[m]);
#pragma unroll
      for (int a = 0; a < 3; a++) {
        lapb[a] = fmaT<T>(wb, vb[a], lapb[a]);
        // d_pa d_pb beta^a: into gdiv[pa] when a == pb, into gdiv[pb] when a == pa != pb
#pragma unroll
        for (int k = 0; k < 3; k++) {
          if (a == pb && k == pa) gdiv[k] = fmaT<T>(sc, vb[a], gdiv[k]);
          if (pa != pb && a == pa && k == pb) gdiv[k] = fmaT<T>(sc, vb[a], gdiv[k]);
        }
      }
    }
  } else {
#pragma unroll
    for (int pa = 0; pa < 3; pa++) {
#pragma unroll
      for (int pb = pa; pb < 3; pb++) {
        const int pq = sym(pa, pb);
        T dd[6];
        T sc;
        if (pa == pb) {
          sc = i12h2;
#pragma unroll
          for (int m = 0; m < 6; m++) dd[m] = d2u<T>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, pa), gt_r[m]);
          ddchi[pq] = d2u<T>(acc, F_CHI, PF(F_CHI), SD(F_CHI, pa), chi_r) * i12h2;
          ddalp[pq] = d2u<T>(acc, F_ALP, PF(F_ALP), SD(F_ALP, pa), alp_r);
        } else if constexpr (XSEG > 0 && !is_f32<T>) {
          if (pa == 0) {
            sc = i12h;
#pragma unroll
            for (int m = 0; m < 6; m++)
              dd[m] = dmx_row<XSEG, YROWS>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, pb), dgt[pb][m], i12h, xep, pb, m);
            ddchi[pq] = dmx_row<XSEG, YROWS>(acc, F_CHI, PF(F_CHI), SD(F_CHI, pb), dchi[pb], i12h, xep, pb, 6) * i12h;
            ddalp[pq] = dmx_row<XSEG, YROWS>(acc, F_ALP, PF(F_ALP), SD(F_ALP, pb), dalp[pb], i12h, xep, pb, 7);
          } else if constexpr (YROWS > 0) {  // (1, 2)
            sc = i12h;
#pragma unroll
            for (int m = 0; m < 6; m++) dd[m] = dyz[m];
            ddchi[pq] = dyz[6] * i12h;
            ddalp[pq] = dyz[7];
          } else {
            sc = i144h2;
#pragma unroll
            for (int m = 0; m < 6; m++) dd[m] = dmu<T>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, pa), SD(F_GT + m, pb));
            ddchi[pq] = dmu<T>(acc, F_CHI, PF(F_CHI), SD(F_CHI, pa), SD(F_CHI, pb)) * i144h2;
            ddalp[pq] = dmu<T>(acc, F_ALP, PF(F_ALP), SD(F_ALP, pa), SD(F_ALP, pb));
          }
        } else {
          sc = i144h2;
#pragma unroll
          for (int m = 0; m < 6; m++) dd[m] = dmu<T>(acc, F_GT + m, PF(F_GT + m), SD(F_GT + m, pa), SD(F_GT + m, pb));
          ddchi[pq] = dmu<T>(acc, F_CHI, PF(F_CHI), SD(F_CHI, pa), SD(F_CHI, pb)) * i144h2;
          ddalp[pq] = dmu<T>(acc, F_ALP, PF(F_ALP), SD(F_ALP, pa), SD(F_ALP, pb));
        }
        sc2[pq] = sc;
        const T wb = sc * g2u[pq];       // gt^{kl} over both orders of (k, l)
        const T w = T(-0.5) * wb;        // -1/2 gt^{kl}
#pragma unroll
        for (int m = 0; m < 6; m++) Rdd[m] = fmaT<T>(w, dd[m], Rdd[m]);
        // shift second derivatives enter the Gt equation even when the shift
        // itself is frozen
#pragma unroll
        for (int a = 0; a < 3; a++) {
          T v;
          if (pa == pb) {
            v = d2u<T>(acc, F_BETA + a, PF(F_BETA + a), SD(F_BETA + a, pa), beta[a]);
          } else if constexpr (XSEG > 0 && !is_f32<T>) {
            if (pa == 0)
              v = dmx_row<XSEG, YROWS>(acc, F_BETA + a, PF(F_BETA + a), SD(F_BETA + a, pb), db[pb][a], i12h, xep,
                                       pb, 8 + a);
            else if constexpr (YROWS > 0)
              v = dyz[8 + a];
            else
              v = dmu<T>(acc, F_BETA + a, PF(F_BETA + a), SD(F_BETA + a, pa), SD(F_BETA + a, pb));
          } else {
            v = dmu<T>(acc, F_BETA + a, PF(F_BETA + a), SD(F_BETA + a, pa), SD(F_BETA + a, pb));
          }
          lapb[a] = fmaT<T>(wb, v, lapb[a]);
          // d_pa d_pb beta^a contributes to gdiv[pa] when a == pb, gdiv[pb] when a == pa
          if (a == pb) gdiv[pa] = fmaT<T>(sc, v, gdiv[pa]);
          if (pa != pb && a == pa) gdiv[pb] = fmaT<T>(sc, v, gdiv[pb]);
        }
      }
    }
  }

  // ---- conformal factor
  T em4, dphi[3], ddphi[6];
  if (g.use_w) {
    const T ih = ihW;
    em4 = chi * chi;
#pragma unroll
    for (int a = 0; a < 3; a++) dphi[a] = -dchi[a] * ih;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++)
        ddphi[sym(a, b)] = fmaT<T>(T(2) * dphi[a], dphi[b], -ddchi[sym(a, b)] * ih);
  } else {
    em4 = expT<T>(T(-4) * chi);
#pragma unroll
    for (int a = 0; a < 3; a++) dphi[a] = dchi[a];
#pragma unroll
    for (int m = 0; m < 6; m++) ddphi[m] = ddchi[m];
  }

  // ---- Christoffel symbols: first kind G1[k][ij] = (d_i g_kj + d_j g_ki - d_k g_ij)/2,
  // with the terms that cancel identically left out (k = i or k = j, i = j)
  T G1[3][6], G2[3][6];
#pragma unroll
  for (int kk = 0; kk < 3; kk++)
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++) {
        T v;
        if (a == b && kk == a)
          v = T(0.5) * dgt[a][sym(a, a)];
        else if (a == b)
          v = fmaT<T>(T(-0.5), dgt[kk][sym(a, a)], dgt[a][sym(kk, a)]);
        else if (kk == a)
          v = T(0.5) * dgt[b][sym(a, a)];
        else if (kk == b)
          v = T(0.5) * dgt[a][sym(b, b)];
        else
          v = T(0.5) * (dgt[a][sym(kk, b)] + dgt[b][sym(kk, a)] - dgt[kk][sym(a, b)]);
        G1[kk][sym(a, b)] = v;
      }
#pragma unroll
  for (int kk = 0; kk < 3; kk++)
#pragma unroll
    for (int m = 0; m < 6; m++)
      G2[kk][m] = gu[sym(kk, 0)] * G1[0][m] + gu[sym(kk, 1)] * G1[1][m] + gu[sym(kk, 2)] * G1[2][m];

  // d_l gt^{lk} = -gt^{kb} (gt^{la} d_l gt_ab)
  T dgu[3];
  {
    T Tb[3];
#pragma unroll
    for (int b = 0; b < 3; b++) {
      T s = T(0);
#pragma unroll
      for (int l = 0; l < 3; l++)
#pragma unroll
        for (int a = 0; a < 3; a++) s = fmaT<T>(gu[sym(l, a)], dgt[l][sym(a, b)], s);
      Tb[b] = s;
    }
#pragma unroll
    for (int kk = 0; kk < 3; kk++)
      dgu[kk] = -(gu[sym(kk, 0)] * Tb[0] + gu[sym(kk, 1)] * Tb[1] + gu[sym(kk, 2)] * Tb[2]);
  }

  // ---- Rt_ij
  T Rt[6];
  {
    // G1u[j][k][l] = gt^{ls} Gt_jks (first kind, last index raised)
    T G1u[3][3][3];
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
        T s = Rdd[ab];
        // gt_k(a d_b) Gt^k + Gt^k Gt_(ab)k with Gt^k = -d_l gt^{lk} and
        // Gt_akb + Gt_bka = d_k gt_ab
        T t = T(0);
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
          t = fmaT<T>(gt[sym(kk, a)], dG[b][kk], t);
          t = fmaT<T>(gt[sym(kk, b)], dG[a][kk], t);
          t = fmaT<T>(-dgt[kk][ab], dgu[kk], t);
        }
        s = fmaT<T>(T(0.5), t, s);
        // gt^{lm} (Gt^k_la Gt_bkm + Gt^k_lb Gt_akm + Gt^k_am Gt_klb); the first
        // two coincide on the diagonal
        if (a == b) {
          T q = T(0);
#pragma unroll
          for (int kk = 0; kk < 3; kk++)
#pragma unroll
            for (int l = 0; l < 3; l++) {
              q = fmaT<T>(G2[kk][sym(l, a)], G1u[a][kk][l], q);
              s = fmaT<T>(G2[kk][sym(a, l)], G1u[kk][a][l], s);
            }
          s = fmaT<T>(T(2), q, s);
        } else {
#pragma unroll
          for (int kk = 0; kk < 3; kk++)
#pragma unroll
            for (int l = 0; l < 3; l++) {
              s = fmaT<T>(G2[kk][sym(l, a)], G1u[b][kk][l], s);
              s = fmaT<T>(G2[kk][sym(l, b)], G1u[a][kk][l], s);
              s = fmaT<T>(G2[kk][sym(a, l)], G1u[kk][b][l], s);
            }
        }
        Rt[ab] = s;
      }
  }

  // ---- Rphi_ij, Dt Dt alpha
  T X[6];
  T lap_alp, dphi_dalp;
  {
    T DDphi[6], DDalp[6];
#pragma unroll
    for (int m = 0; m < 6; m++) {
      DDphi[m] = ddphi[m] - (G2[0][m] * dphi[0] + G2[1][m] * dphi[1] + G2[2][m] * dphi[2]);
      DDalp[m] = fmaT<T>(sc2[m], ddalp[m], -(G2[0][m] * dalp[0] + G2[1][m] * dalp[1] + G2[2][m] * dalp[2]));
    }
    T lap_phi = T(0);
    lap_alp = T(0);
#pragma unroll
    for (int m = 0; m < 6; m++) {
      lap_phi = fmaT<T>(g2u[m], DDphi[m], lap_phi);
      lap_alp = fmaT<T>(g2u[m], DDalp[m], lap_alp);
    }
    T uphi[3];  // gt^{ab} d_b phi
#pragma unroll
    for (int a = 0; a < 3; a++) uphi[a] = gu[sym(a, 0)] * dphi[0] + gu[sym(a, 1)] * dphi[1] + gu[sym(a, 2)] * dphi[2];
    const T grad2 = uphi[0] * dphi[0] + uphi[1] * dphi[1] + uphi[2] * dphi[2];
    dphi_dalp = uphi[0] * dalp[0] + uphi[1] * dalp[1] + uphi[2] * dalp[2];
    // Rphi_ab = -2 DD_ab phi + 4 d_a phi d_b phi - gt_ab (2 lap phi + 4 |d phi|^2)
    const T cg = fmaT<T>(T(4), grad2, T(2) * lap_phi);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++) {
        const int ab = sym(a, b);
        const T rphi = fmaT<T>(T(-2), DDphi[ab], fmaT<T>(T(4) * dphi[a], dphi[b], -gt[ab] * cg));
        const T cross = fmaT<T>(dphi[a], dalp[b], dphi[b] * dalp[a]);
        X[ab] = fmaT<T>(T(2), cross, fmaT<T>(alp, Rt[ab] + rphi, -DDalp[ab]));
      }
  }

  // ---- At with raised indices
  T Aud[3][3], Auu[6], Auu2[6];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++)
      Aud[a][b] = gu[sym(a, 0)] * At[sym(0, b)] + gu[sym(a, 1)] * At[sym(1, b)] +
                  gu[sym(a, 2)] * At[sym(2, b)];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = a; b < 3; b++)
      Auu[sym(a, b)] = Aud[a][0] * gu[sym(0, b)] + Aud[a][1] * gu[sym(1, b)] + Aud[a][2] * gu[sym(2, b)];
#pragma unroll
  for (int m = 0; m < 6; m++) Auu2[m] = (m == 0 || m == 3 || m == 5) ? Auu[m] : T(2) * Auu[m];
  T AA = T(0);
#pragma unroll
  for (int m = 0; m < 6; m++) AA = fmaT<T>(Auu2[m], At[m], AA);
  const T divb = db[0][0] + db[1][1] + db[2][2];

  // ---- matter sources, when a stress-energy tensor is given: the paper's
  // -alpha S, -alpha e^{-4 phi} Shat_ij and -S^i in the normalisation G = 8 pi T,
  // i.e. d_0 K += 4 pi alpha (E + S), d_0 At_ij -= 8 pi alpha e^{-4 phi} [S_ij]^TF,
  // d_0 Gt^i -= 16 pi alpha gt^ij S_j (and the Gamma-driver through d_0 Gt^i)
  const bool matter = g.tmunu != nullptr;
  T mK = T(0), mA = T(0), mG[3] = {T(0), T(0), T(0)}, Stf[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  if (matter) {
    T Em, Smi[3];
    matter_at<T>(g, lin(g, i, j, k), alp, beta, Em, Smi, Stf);
    T trs = T(0);
#pragma unroll
    for (int m = 0; m < 6; m++) trs = fmaT<T>(g2u[m], Stf[m], trs);
#pragma unroll
    for (int m = 0; m < 6; m++) Stf[m] -= gt[m] * trs * T(1.0 / 3.0);  // [S_ij]^TF (gt_ij gt^kl = gamma_ij gamma^kl)
    mK = T(4.0 * M_PI) * alp * (Em + em4 * trs);
    mA = T(-8.0 * M_PI) * alp * em4;
#pragma unroll
    for (int a = 0; a < 3; a++)
      mG[a] = T(-16.0 * M_PI) * alp * (gu[sym(a, 0)] * Smi[0] + gu[sym(a, 1)] * Smi[1] + gu[sym(a, 2)] * Smi[2]);
  }

  // ---- assemble
  if (g.use_w)
    out[F_CHI] = (chi * T(1.0 / 3.0)) * (alp * trK - divb);
  else
    out[F_CHI] = T(-1.0 / 6.0) * alp * trK + divb * T(1.0 / 6.0);

  const T divb23 = T(2.0 / 3.0) * divb;
  {
    T trX = T(0);
#pragma unroll
    for (int m = 0; m < 6; m++) trX = fmaT<T>(g2u[m], X[m], trX);
    const T trX3 = trX * T(1.0 / 3.0);
    const T akd = fmaT<T>(alp, trK, -divb23);  // alpha K - 2/3 d_k beta^k
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++) {
        const int ab = sym(a, b);
        T sg = T(-2) * alp * At[ab] - gt[ab] * divb23;
        T sa = fmaT<T>(akd, At[ab], em4 * fmaT<T>(-gt[ab], trX3, X[ab]));
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
          sg = fmaT<T>(gt[sym(kk, a)], db[b][kk], sg);
          sg = fmaT<T>(gt[sym(kk, b)], db[a][kk], sg);
          sa = fmaT<T>(T(-2) * alp * At[sym(a, kk)], Aud[kk][b], sa);
          sa = fmaT<T>(At[sym(kk, a)], db[b][kk], sa);
          sa = fmaT<T>(At[sym(kk, b)], db[a][kk], sa);
        }
        out[F_GT + ab] = sg;
        out[F_AT + ab] = matter ? fmaT<T>(mA, Stf[ab], sa) : sa;
      }
  }

  out[F_TRK] = -em4 * (lap_alp + T(2) * dphi_dalp) + alp * (AA + trK * trK * T(1.0 / 3.0)) + mK;

  T gam_rhs[3];
  {
    // -2 At^{aj} d_j alpha + 12 alpha At^{aj} d_j phi = At^{aj} vj_j
    T vj[3], dKu[3], gdu[3];
    const T a12 = T(12) * alp;
#pragma unroll
    for (int jj = 0; jj < 3; jj++) vj[jj] = fmaT<T>(a12, dphi[jj], T(-2) * dalp[jj]);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      dKu[a] = gu[sym(a, 0)] * dK[0] + gu[sym(a, 1)] * dK[1] + gu[sym(a, 2)] * dK[2];
      gdu[a] = gu[sym(a, 0)] * gdiv[0] + gu[sym(a, 1)] * gdiv[1] + gu[sym(a, 2)] * gdiv[2];
    }
    const T m23divb = T(-2.0 / 3.0) * divb;
    const T alp2 = T(2) * alp;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      T s = fmaT<T>(T(1.0 / 3.0), gdu[a], lapb[a]);
      s = fmaT<T>(dgu[0], db[0][a], s);
      s = fmaT<T>(dgu[1], db[1][a], s);
      s = fmaT<T>(dgu[2], db[2][a], s);
      s = fmaT<T>(m23divb, dgu[a], s);
#pragma unroll
      for (int jj = 0; jj < 3; jj++) s = fmaT<T>(Auu[sym(a, jj)], vj[jj], s);
      // Gt^a_kl At^kl - 2/3 gt^aj d_j K
      T br = T(-2.0 / 3.0) * dKu[a];
#pragma unroll
      for (int m = 0; m < 6; m++) br = fmaT<T>(G2[a][m], Auu2[m], br);
      s = fmaT<T>(alp2, br, s);
      if (matter) s += mG[a];
      gam_rhs[a] = s;
      out[F_GAM + a] = s;
    }
  }

  if (g.slicing == BSSN_1PLUSLOG)
    out[F_ALP] = T(-2) * alp * trK;
  else if (g.slicing == BSSN_HARMONIC)
    out[F_ALP] = -alp * alp * trK;
  else
    out[F_ALP] = T(0);

  const bool frozen = (g.shift == BSSN_SHIFT_FROZEN);
  if (!frozen) {
    T q = T(1);
    if (g.q_R > 0.0 && !isinf(g.q_R)) {
      double x = g.xmin0 + (i - GH + 0.5) * g.h, y = g.xmin1 + (j - GH + 0.5) * g.h,
             z = g.xmin2 + (k - GH + 0.5) * g.h;
      double r = sqrt(x * x + y * y + z * z);
      q = r <= g.q_R ? T(1) : T(g.q_R / r);
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
      out[F_BETA + a] = T(0.75) * Bv[a];
      out[F_B + a] = gam_rhs[a] - gc<T>(g.eta, g.etaf, g.etal) * q * Bv[a];
    }
  }

  // ---- advection and dissipation, every field (one weighted stencil per axis)
  const int nf = frozen ? F_BETA : NF;
#pragma unroll
  for (int f = F_BETA; f < NF; f++)
    if (f >= nf) out[f] = T(0);
  if constexpr (is_precomputed<A>::value) {
#pragma unroll
    for (int f = 0; f < NF; f++)
      if (f < nf) out[f] += acc.template advko<T>(f);
  } else if constexpr (ROLL) {
    // one loop over the fields: the same weights and the same order of
    // accumulation as below (centre term, then axes x, y, z, offsets -3..3)
    const T kap = gc<T>(g.kos, g.kosf, g.kosl);
    T bh[3];
#pragma unroll
    for (int d = 0; d < 3; d++) bh[d] = absT<T>(beta[d]) * i12h;
    const T w0 = fmaT<T>(T(-10), bh[0] + bh[1] + bh[2], T(-60) * kap);
    const T cko[7] = {T(1), T(-6), T(15), T(-20), T(15), T(-6), T(1)};
    T w[3][7];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const bool pos = beta[d] >= T(0);
#pragma unroll
      for (int m = -3; m <= 3; m++)
        if (m != 0) w[d][m + 3] = fmaT<T>(bh[d], up_coefT<T>(pos, m), kap * cko[m + 3]);
    }
    T r[NF];  // indexed at run time
#pragma unroll
    for (int f = 0; f < NF; f++) r[f] = out[f];
    const long long s3[3] = {SD(F_GT, 0), SD(F_GT, 1), SD(F_GT, 2)};
#pragma unroll 1
    for (int f = 0; f < nf; f++) {
      const auto* p = PF(f);
      T accv = fmaT<T>(w0, LD(f, p), r[f]);
#pragma unroll
      for (int d = 0; d < 3; d++)
#pragma unroll
        for (int m = -3; m <= 3; m++)
          if (m != 0) accv = fmaT<T>(w[d][m + 3], LD(f, p + m * s3[d]), accv);
      r[f] = accv;
    }
#pragma unroll
    for (int f = 0; f < NF; f++) out[f] = r[f];
  } else {
    const T kap = gc<T>(g.kos, g.kosf, g.kosl);
    T f0s[NF];  // centre values as stored (float: the stencil is applied to f_m - f0)
    T bh[3];
#pragma unroll
    for (int d = 0; d < 3; d++) bh[d] = absT<T>(beta[d]) * i12h;
    const T w0 = fmaT<T>(T(-10), bh[0] + bh[1] + bh[2], T(-60) * kap);
#pragma unroll
    for (int f = 0; f < NF; f++) {
      if (f >= nf) break;
      T f0;  // as stored: the stencil weights apply to stored values
      if (f == F_CHI) f0 = chi_r;
      else if (f >= F_GT && f < F_GT + 6) f0 = gt_r[f - F_GT];
      else if (f == F_TRK) f0 = trK;
      else if (f >= F_AT && f < F_AT + 6) f0 = At[f - F_AT];
      else if (f == F_ALP) f0 = alp_r;
      else if (f >= F_BETA && f < F_BETA + 3) f0 = beta[f - F_BETA];
      else if (f >= F_B) f0 = Bv[f - F_B];
      else f0 = LD(f, PF(f));
      if constexpr (!is_f32<T>) out[f] = fmaT<T>(w0, f0, out[f]);
      f0s[f] = f0;
    }
    const T cko[7] = {T(1), T(-6), T(15), T(-20), T(15), T(-6), T(1)};
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const bool pos = beta[d] >= T(0);
      T w[7];
#pragma unroll
      for (int m = -3; m <= 3; m++)
        if (m != 0) w[m + 3] = fmaT<T>(bh[d], up_coefT<T>(pos, m), kap * cko[m + 3]);
#pragma unroll
      for (int f = 0; f < NF; f++) {
        if (f >= nf) break;
        const auto* p = PF(f);
        T accv = out[f];
        if constexpr (is_f32<T>) {
          // the weights sum to zero: apply them to differences to the centre
#pragma unroll
          for (int m = -3; m <= 3; m++)
            if (m != 0) accv = fmaT<T>(w[m + 3], LD(f, p + m * SD(f, d)) - f0s[f], accv);
        } else {
#pragma unroll
          for (int m = -3; m <= 3; m++)
            if (m != 0) accv = fmaT<T>(w[m + 3], LD(f, p + m * SD(f, d)), accv);
        }
        out[f] = accv;
      }
    }
  }
#undef PF
#undef SD
#undef LD
}

// Right-hand side reading every field from the global register st.
template <typename T, typename S, bool DEV = false, int XSEG = 0, int YROWS = 0, int ZS = 1>
__device__ __forceinline__ void rhs_point(const Grid& g, const S* __restrict__ st, long long id,
                                          int i, int j, int k, T out[NF]) {
  const GlobalAcc<S> acc(g, st, id);
  rhs_point_acc<T, S, DEV, GlobalAcc<S>, XSEG, YROWS, ZS>(g, acc, i, j, k, out);
}

}  // namespace bssn
