// Fused BSSN right-hand side + RK4 stage combination.
//
// One thread per interior point.  The right-hand side (rhs_point.cuh) is
// evaluated from the stage input register and combined at once with y_n and
// the k-sum, so k is never stored except at the interior points next to
// the outer boundary, whose k the Sommerfeld boundary needs (anchor buffer).
// Classical RK4 (the method of lines that evolves the equations of Sec.
// "Spacetime Curvature Evolution") with registers y_n, ks (k-sum) and two
// stage buffers, y_n advanced in place:
//   stage 1: s1 = y + dt/2 k1,  ks = k1
//   stage 2: s2 = y + dt/2 k2,  ks += 2 k2
//   stage 3: s1 = y + dt k3,    ks += 2 k3
//   stage 4: y += dt/6 (ks + k4)
//
// Float64 path: everything in double.  Mixed path: the state y_n stays in
// double and is advanced once per step, y_{n+1} = y_n + dt/6 (k1 + 2k2 + 2k3
// + k4), in double; the stage values y_n + c dt k are formed in float from a
// float shadow of y_n (they are stored in float anyway) and the weighted sum
// of the k in float; stencils and right-hand side run in float.  W is carried
// in double alongside every float stage buffer, its stage values and k-sum are
// double, and where W is below the threshold (near a puncture) its
// right-hand side is recomputed in double from that double W.  This keeps the
// float<->double conversions, which share the slow float64 pipe, to one pair
// per field per step.
#include "stage_point.cuh"

namespace bssn {

// One thread per interior point; TX x TY x TZ points per block.
template <int TX, int TY, int TZ, int MINB>
__global__ void __launch_bounds__(TX * TY * TZ, MINB) stage_fp64_kernel(Grid g, StageArgs a) {
  const int ii = blockIdx.x * TX + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  stage_point_fp64<0>(g, a, ii, jj, kk);
}

template <int TX, int TY, int TZ, int MINB, bool KS64 = false>
__global__ void __launch_bounds__(TX * TY * TZ, MINB) stage_mixed_kernel(Grid g, StageArgsMixed a) {
  const int ii = blockIdx.x * TX + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  stage_point_mixed<KS64>(g, a, ii, jj, kk);
}

// float64 full-row variants, defined in k_stage_shfl.cu
template <int TY, int TZ, int MINB>
cudaError_t launch_fp64_rows(const Grid& g, const StageArgs& a, cudaStream_t s);
extern template cudaError_t launch_fp64_rows<8, 1, 1>(const Grid&, const StageArgs&, cudaStream_t);
extern template cudaError_t launch_fp64_rows<4, 1, 1>(const Grid&, const StageArgs&, cudaStream_t);
extern template cudaError_t launch_fp64_rows<4, 2, 1>(const Grid&, const StageArgs&, cudaStream_t);
extern template cudaError_t launch_fp64_rows<2, 2, 2>(const Grid&, const StageArgs&, cudaStream_t);

// ------------------------------------------------------ tile configurations
// Candidate block shapes (points per block along x, y, z) and the minimum
// resident blocks per SM handed to the compiler (which caps registers and so
// trades spills for occupancy).  The autotuner times them on the live state.
template <int TX, int TY, int TZ, int MINB>
static cudaError_t launch_fp64_t(const Grid& g, const StageArgs& a, cudaStream_t s) {
  dim3 block(TX, TY, TZ);
  dim3 grid((g.n0 + TX - 1) / TX, (g.n1 + TY - 1) / TY, (g.n2 + TZ - 1) / TZ);
  stage_fp64_kernel<TX, TY, TZ, MINB><<<grid, block, 0, s>>>(g, a);
  return cudaGetLastError();
}
template <int TX, int TY, int TZ, int MINB>
static cudaError_t launch_mixed_t(const Grid& g, const StageArgsMixed& a, cudaStream_t s) {
  dim3 block(TX, TY, TZ);
  dim3 grid((g.n0 + TX - 1) / TX, (g.n1 + TY - 1) / TY, (g.n2 + TZ - 1) / TZ);
  stage_mixed_kernel<TX, TY, TZ, MINB><<<grid, block, 0, s>>>(g, a);
  return cudaGetLastError();
}

struct TileCfg {
  const char* name;
  cudaError_t (*fp64)(const Grid&, const StageArgs&, cudaStream_t);
  cudaError_t (*mixed)(const Grid&, const StageArgsMixed&, cudaStream_t);
  // float64 variant whose warps are full 32-point x-rows sharing first
  // differences (k_stage_shfl.cu); used when n0 is a multiple of 32
  cudaError_t (*fp64_rows)(const Grid&, const StageArgs&, cudaStream_t);
};

#define TILE(TX, TY, TZ, MINB)                                                  \
  { #TX "x" #TY "x" #TZ "/" #MINB, launch_fp64_t<TX, TY, TZ, MINB>,            \
    launch_mixed_t<TX, TY, TZ, MINB>, nullptr }
#define TILE_ROWS(TY, TZ, MINB)                                                 \
  { "32x" #TY "x" #TZ "/" #MINB, launch_fp64_t<32, TY, TZ, MINB>,              \
    launch_mixed_t<32, TY, TZ, MINB>, launch_fp64_rows<TY, TZ, MINB> }
// mixed only: registers capped for four or six resident blocks per SM (more
// warps to cover the load latency, more spills)
#define TILE_MX(TX, TY, TZ, MINB) \
  { #TX "x" #TY "x" #TZ "/" #MINB, nullptr, launch_mixed_t<TX, TY, TZ, MINB>, nullptr }
static const TileCfg k_tiles[] = {
    TILE_ROWS(8, 1, 1), TILE_ROWS(4, 1, 1), TILE_ROWS(4, 2, 1), TILE(64, 4, 1, 1),
    TILE(16, 8, 2, 1), TILE_ROWS(2, 2, 2), TILE(32, 8, 1, 2), TILE(32, 4, 1, 3),
    TILE_MX(32, 4, 1, 4), TILE_MX(32, 4, 1, 6),
};
#undef TILE_MX
#undef TILE
#undef TILE_ROWS

int tile_config_count() { return (int)(sizeof(k_tiles) / sizeof(k_tiles[0])); }
bool tile_config_has_fp64(int c) { return c >= 0 && c < tile_config_count() && k_tiles[c].fp64 != nullptr; }
const char* tile_config_name(int c) {
  return (c >= 0 && c < tile_config_count()) ? k_tiles[c].name : "";
}

cudaError_t launch_stage_fp64(const Grid& g, const StageArgs& a, cudaStream_t s, int cfg) {
  if (!tile_config_has_fp64(cfg)) cfg = 0;
  if (k_tiles[cfg].fp64_rows && g.n0 % 32 == 0) return k_tiles[cfg].fp64_rows(g, a, s);
  return k_tiles[cfg].fp64(g, a, s);
}

cudaError_t launch_stage_mixed(const Grid& g, const StageArgsMixed& a, cudaStream_t s, int cfg) {
  if (cfg < 0 || cfg >= tile_config_count()) cfg = 0;
  return k_tiles[cfg].mixed(g, a, s);
}

// the mixed stage with the float64 k-sum of every field (ksum_fp64): the fused
// 32 x 8 x 1 kernel, whatever the context's tile configuration
cudaError_t launch_stage_mixed_ks64(const Grid& g, const StageArgsMixed& a, cudaStream_t s) {
  dim3 block(32, 8, 1);
  dim3 grid((g.n0 + 31) / 32, (g.n1 + 7) / 8, g.n2);
  stage_mixed_kernel<32, 8, 1, 1, true><<<grid, block, 0, s>>>(g, a);
  return cudaGetLastError();
}

// float shadow X - X0 (and float64 W) of a float64 register, every stored point
__global__ void shadow_kernel(Grid g, const double* __restrict__ y, float* __restrict__ s32,
                              double* __restrict__ w) {
  const long long n = (long long)NF * g.fstride;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double v = y[q];
    s32[q] = (float)(v - background(g, (int)(q / g.fstride)));
    if (q < g.fstride) w[q] = v;
  }
}

cudaError_t launch_shadow(const Grid& g, const double* y, float* s32, double* w, cudaStream_t s) {
  shadow_kernel<<<152 * 8, 256, 0, s>>>(g, y, s32, w);
  return cudaGetLastError();
}

}  // namespace bssn
