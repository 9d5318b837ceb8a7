// Mixed-precision stage split into a stencil pass and an algebra pass.
//
// The fused mixed stage (k_stage.cu, k_stage_tma.cu) evaluates about 1200
// stencil reads and the whole right-hand side algebra in one thread; at 255
// registers only 8 warps fit on an SM and the kernel waits on its loads.  Here
//  1. deriv_kernel, one thread per (point, field), forms every difference the
//     right-hand side uses -- 45 first differences (phi|W, gt_ij, K, Gt^i,
//     alpha, beta^i), 66 second differences (phi|W, gt_ij, alpha, beta^i) and
//     the upwinded-advection + Kreiss-Oliger sum of all 24 fields -- with the
//     same float operations as the fused kernel, into a derivative register
//     of NSLOT float fields;
//  2. stage_split_kernel runs the same per-point stage (stage_point.cuh) with
//     an accessor that returns those values instead of applying stencils.
// The differences are the fused kernel's bits (same operations, stored and
// reloaded exactly); only the order in which the advection/dissipation sum
// joins the right-hand side differs (float rounding).
#include "stage_point.cuh"

namespace bssn {

namespace {

// slots of the derivative register
__host__ __device__ constexpr int d1_index(int f) {  // fields with first differences
  return f == F_CHI ? 0
         : (f >= F_GT && f < F_GT + 6) ? 1 + (f - F_GT)
         : f == F_TRK ? 7
         : (f >= F_GAM && f < F_GAM + 3) ? 8 + (f - F_GAM)
         : f == F_ALP ? 11
         : (f >= F_BETA && f < F_BETA + 3) ? 12 + (f - F_BETA)
                                          : -1;
}
__host__ __device__ constexpr int d2_index(int f) {  // fields with second differences
  return f == F_CHI ? 0
         : (f >= F_GT && f < F_GT + 6) ? 1 + (f - F_GT)
         : f == F_ALP ? 7
         : (f >= F_BETA && f < F_BETA + 3) ? 8 + (f - F_BETA)
                                          : -1;
}
constexpr int ND1 = 15, ND2 = 11;
constexpr int SLOT_D1 = 0;                     // + 3 d1_index(f) + d
constexpr int SLOT_D2 = SLOT_D1 + 3 * ND1;     // + 6 d2_index(f) + sym(a, b)
constexpr int SLOT_AK = SLOT_D2 + 6 * ND2;     // + f
constexpr int NSLOT_ = SLOT_AK + NF;           // 135

}  // namespace

// Accessor of the algebra pass: field values from the stage input, differences
// and advection/dissipation sums from the derivative register.  s(f, d)
// returns the axis d itself in place of a stride; the difference overloads
// below map (field, axis) to the slot.
struct DerivAcc {
  const float* __restrict__ st;
  const float* __restrict__ dr;
  long long id, fs;
  __device__ __forceinline__ const float* ptr(int f) const { return st + (long long)f * fs + id; }
  __device__ __forceinline__ long long s(int, int d) const { return d; }
  template <typename T>
  __device__ __forceinline__ T ld(int, const float* p) const { return T(__ldg(p)); }
  __device__ __forceinline__ float slot(int q) const { return __ldg(dr + (long long)q * fs + id); }
  template <typename T>
  __device__ __forceinline__ T advko(int f) const { return T(slot(SLOT_AK + f)); }
};
template <>
struct is_precomputed<DerivAcc> {
  static constexpr bool value = true;
};
template <typename T, typename P>
__device__ __forceinline__ T d1u(const DerivAcc& a, int f, const P*, long long d) {
  return T(a.slot(SLOT_D1 + 3 * d1_index(f) + (int)d));
}
template <typename T, typename P>
__device__ __forceinline__ T d2u(const DerivAcc& a, int f, const P*, long long d, T) {
  return T(a.slot(SLOT_D2 + 6 * d2_index(f) + sym((int)d, (int)d)));
}
template <typename T, typename P>
__device__ __forceinline__ T dmu(const DerivAcc& a, int f, const P*, long long da, long long db) {
  return T(a.slot(SLOT_D2 + 6 * d2_index(f) + sym((int)da, (int)db)));
}

int split_slot_count() { return NSLOT_; }

namespace {

constexpr int DX = 32, DY = 4;  // deriv_kernel block: 32 x 4 points of one field

__global__ void __launch_bounds__(DX * DY) deriv_kernel(Grid g, const float* __restrict__ st,
                                                        float* __restrict__ dr) {
  const int f = blockIdx.z;
  const int nty = (g.n1 + DY - 1) / DY;
  const int ii = blockIdx.x * DX + threadIdx.x;
  const int jj = (blockIdx.y % nty) * DY + threadIdx.y;
  const int kk = blockIdx.y / nty;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  const long long fs = g.fstride;
  const long long id = lin(g, ii + GH, jj + GH, kk + GH);
  const long long sd[3] = {1, g.pitch, g.plane};
  const float* p = st + (long long)f * fs + id;
  float* o = dr + id;
  const float f0 = __ldg(p);
  const PlainAcc<float, float> pa{};
  const int i1 = d1_index(f), i2 = d2_index(f);
  if (i1 >= 0) {
#pragma unroll
    for (int d = 0; d < 3; d++) o[(SLOT_D1 + 3 * i1 + d) * fs] = d1u<float>(pa, f, p, sd[d]);
  }
  if (i2 >= 0) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = a; b < 3; b++)
        o[(SLOT_D2 + 6 * i2 + sym(a, b)) * fs] =
            a == b ? d2u<float>(pa, f, p, sd[a], f0) : dmu<float>(pa, f, p, sd[a], sd[b]);
  }
  // upwinded advection + KO dissipation, as the fused kernel forms it in float:
  // sum_d sum_{m != 0} w_d[m] (f_m - f_0)
  const float i12h = g.i12hf, kap = g.kosf;
  const float cko[7] = {1.f, -6.f, 15.f, -20.f, 15.f, -6.f, 1.f};
  float acc = 0.f;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const float bd = __ldg(st + (long long)(F_BETA + d) * fs + id);
    const float bh = fabsf(bd) * i12h;
    const bool pos = bd >= 0.f;
#pragma unroll
    for (int m = -3; m <= 3; m++)
      if (m != 0) acc = fmaf(fmaf(bh, float(up_coef(pos, m)), kap * cko[m + 3]), __ldg(p + m * sd[d]) - f0, acc);
  }
  o[(SLOT_AK + f) * fs] = acc;
}

template <int TX, int TY, int TZ, int MINB>
__global__ void __launch_bounds__(TX * TY * TZ, MINB)
    stage_split_kernel(Grid g, StageArgsMixed a, const float* __restrict__ dr) {
  const int ii = blockIdx.x * TX + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  const DerivAcc acc{a.src, dr, lin(g, ii + GH, jj + GH, kk + GH), g.fstride};
  stage_point_mixed_acc(g, a, acc, ii, jj, kk);
}

// algebra-pass variants: block shape and minimum resident blocks per SM (the
// register budget: 2 -> 255, 3 -> 168, 4 -> 128 registers for 128 threads)
struct SplitCfg {
  const char* name;
  int tx, ty, tz;
  const void* fn;
};
#define SCFG(TX, TY, TZ, MINB) \
  { "split" #TX "x" #TY "x" #TZ "/" #MINB, TX, TY, TZ, (const void*)stage_split_kernel<TX, TY, TZ, MINB> }
const SplitCfg k_split[] = {SCFG(32, 4, 1, 2), SCFG(32, 4, 1, 3), SCFG(32, 4, 1, 4)};
#undef SCFG

}  // namespace

int split_config_count() { return (int)(sizeof(k_split) / sizeof(k_split[0])); }
const char* split_config_name(int v) { return (v >= 0 && v < split_config_count()) ? k_split[v].name : ""; }

cudaError_t launch_stage_mixed_split(const Grid& g, const StageArgsMixed& a, float* dr, cudaStream_t s,
                                     int variant) {
  if (variant < 0 || variant >= split_config_count()) variant = 0;
  const int nty = (g.n1 + DY - 1) / DY;
  if ((long long)nty * g.n2 > 65535) return cudaErrorInvalidConfiguration;  // grid y limit
  dim3 dgrid((g.n0 + DX - 1) / DX, nty * g.n2, NF);
  deriv_kernel<<<dgrid, dim3(DX, DY), 0, s>>>(g, a.src, dr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const SplitCfg& c = k_split[variant];
  dim3 rgrid((g.n0 + c.tx - 1) / c.tx, (g.n1 + c.ty - 1) / c.ty, (g.n2 + c.tz - 1) / c.tz);
  const Grid* gp = &g;
  const StageArgsMixed* ap = &a;
  const float* drc = dr;
  void* args[] = {(void*)gp, (void*)ap, (void*)&drc};
  return cudaLaunchKernel(c.fn, rgrid, dim3(c.tx, c.ty, c.tz), args, 0, s);
}

}  // namespace bssn
