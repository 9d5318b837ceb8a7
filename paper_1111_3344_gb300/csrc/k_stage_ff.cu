// Double-word precision path: the fused BSSN right-hand side + RK4 stage with
// the stencils and the right-hand side in double-word ("float-float")
// arithmetic on the float32 pipe (ff.cuh), and the RK4 state y_n and the
// weighted sum of the k in float64.
//
// The right-hand side is the same per-point code as the other paths
// (rhs_point.cuh, the equations of Sec. "Spacetime Curvature Evolution"),
// instantiated with the double-word type and reading the stage buffers as
// double-word values {hi, lo} of X (8 bytes a value, as on the float64 path).
// Classical RK4 with y_n advanced in place once per step:
//   stage 1: s1 = y + dt/2 k1,  ks = k1          (s0: double-word shadow of y_n)
//   stage 2: s2 = y + dt/2 k2,  ks += 2 k2
//   stage 3: s1 = y + dt k3,    ks += 2 k3
//   stage 4: y += dt/6 (ks + k4), s0 = shadow of the new y
// The stage values are formed in double-word arithmetic from the shadow; the
// k-sum and the update of y_n are float64 (one float64 conversion of each k).
// The Sommerfeld boundary (Sec. "Boundary Conditions") runs in float64
// arithmetic on the double-word stage values, one thread per ghost point.
#include "boundary_point.cuh"
#include "stage_point.cuh"

namespace bssn {

template <int TX, int TY, int TZ, int MINB>
__global__ void __launch_bounds__(TX * TY * TZ, MINB) stage_ff_kernel(Grid g, StageArgsFF a) {
  const int ii = blockIdx.x * TX + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  stage_point_ff(g, a, ii, jj, kk);
}

__global__ void sommerfeld_ff_kernel(Grid g, StageArgsFF a, const float2* __restrict__ kanchor) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ghost_count(g)) return;
  sommerfeld_point_ff(g, a, kanchor, q);
}

// double-word shadow {hi, lo} of a float64 register, every stored point
__global__ void shadow_ff_kernel(Grid g, const double* __restrict__ y, float2* __restrict__ s2) {
  const long long n = (long long)NF * g.fstride;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    s2[q] = ff_from_double(y[q]).f2();
}

// ------------------------------------------------------ configurations
// full-row and full-block variants (k_stage_ff_rows.cu)
template <int TY, int TZ, int MINB>
cudaError_t launch_ff_rows(const Grid& g, const StageArgsFF& a, cudaStream_t s);
extern template cudaError_t launch_ff_rows<4, 1, 1>(const Grid&, const StageArgsFF&, cudaStream_t);
extern template cudaError_t launch_ff_rows<8, 1, 1>(const Grid&, const StageArgsFF&, cudaStream_t);
extern template cudaError_t launch_ff_rows<4, 2, 1>(const Grid&, const StageArgsFF&, cudaStream_t);
extern template cudaError_t launch_ff_rows<4, 1, 3>(const Grid&, const StageArgsFF&, cudaStream_t);
extern template cudaError_t launch_ff_rows<4, 1, 4>(const Grid&, const StageArgsFF&, cudaStream_t);
extern template cudaError_t launch_ff_rows<4, 1, 5>(const Grid&, const StageArgsFF&, cudaStream_t);
extern template cudaError_t launch_ff_rows<4, 1, 6>(const Grid&, const StageArgsFF&, cudaStream_t);
extern template cudaError_t launch_ff_rows<4, 1, 8>(const Grid&, const StageArgsFF&, cudaStream_t);

template <int TX, int TY, int TZ, int MINB>
static cudaError_t launch_ff_t(const Grid& g, const StageArgsFF& a, cudaStream_t s) {
  dim3 block(TX, TY, TZ);
  dim3 grid((g.n0 + TX - 1) / TX, (g.n1 + TY - 1) / TY, (g.n2 + TZ - 1) / TZ);
  stage_ff_kernel<TX, TY, TZ, MINB><<<grid, block, 0, s>>>(g, a);
  return cudaGetLastError();
}

struct FfCfg {
  const char* name;
  cudaError_t (*launch)(const Grid&, const StageArgsFF&, cudaStream_t);
};
#define FF_TILE(TX, TY, TZ, MINB) {"ff" #TX "x" #TY "x" #TZ "/" #MINB, launch_ff_t<TX, TY, TZ, MINB>}
#define FF_ROWS(TY, TZ, MINB) {"ffrows32x" #TY "x" #TZ "/" #MINB, launch_ff_rows<TY, TZ, MINB>}
static const FfCfg k_ff[] = {
    FF_ROWS(4, 1, 1), FF_ROWS(8, 1, 1), FF_ROWS(4, 2, 1), FF_ROWS(4, 1, 3), FF_ROWS(4, 1, 4),
    FF_ROWS(4, 1, 5), FF_ROWS(4, 1, 6), FF_ROWS(4, 1, 8), FF_TILE(32, 4, 1, 1),
};
#undef FF_TILE
#undef FF_ROWS

int ff_config_count() { return (int)(sizeof(k_ff) / sizeof(k_ff[0])); }
const char* ff_config_name(int c) { return (c >= 0 && c < ff_config_count()) ? k_ff[c].name : ""; }

// the every-stencil kernel for grids whose n0 is not a multiple of 32 (the
// row variants' fallback)
cudaError_t launch_ff_any(const Grid& g, const StageArgsFF& a, cudaStream_t s) {
  return launch_ff_t<32, 4, 1, 1>(g, a, s);
}

cudaError_t launch_stage_ff(const Grid& g, const StageArgsFF& a, cudaStream_t s, int cfg) {
  if (cfg < 0 || cfg >= ff_config_count()) cfg = 0;
  return k_ff[cfg].launch(g, a, s);
}

cudaError_t launch_sommerfeld_ff(const Grid& g, const StageArgsFF& a, const float2* kanchor, cudaStream_t s) {
  const unsigned total = ghost_count(g);
  const int bs = 128;
  sommerfeld_ff_kernel<<<(total + bs - 1) / bs, bs, 0, s>>>(g, a, kanchor);
  return cudaGetLastError();
}

cudaError_t launch_shadow_ff(const Grid& g, const double* y, float2* s2, cudaStream_t s) {
  shadow_ff_kernel<<<152 * 8, 256, 0, s>>>(g, y, s2);
  return cudaGetLastError();
}

}  // namespace bssn
