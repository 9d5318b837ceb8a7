// Float64 fused stage for blocks whose warps are full rows of 32 x points
// (n0 a multiple of 32, TX = 32): the mixed second differences D1_x D1_y and
// D1_x D1_z take the neighbouring points' first differences along y or z from
// the neighbouring lanes (dmx_shfl in rhs_point.cuh) instead of evaluating
// four more first differences per field.  Everything else is the stage of
// k_stage.cu; a warp is either wholly inside the grid or wholly outside it
// (rows past n1 or n2), so the shuffles always see 32 active lanes.
#include "stage_point.cuh"

namespace bssn {

template <int TY, int TZ, int MINB>
__global__ void __launch_bounds__(32 * TY * TZ, MINB) stage_fp64_rows_kernel(Grid g, StageArgs a) {
  const int ii = blockIdx.x * 32 + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  if (jj >= g.n1 || kk >= g.n2) return;  // whole warps
  stage_point_fp64<32>(g, a, ii, jj, kk);
}

// Full blocks (n1 % TY == 0 and n2 % TZ == 0 as well): every thread is inside
// the grid, so the block can also exchange first differences along z through
// shared memory for D_y D_z, and each warp's 32 lanes form the first
// differences past the ends of its row that D_x D_y and D_x D_z need, into
// shared memory, instead of the two lanes at each end (dmx_pre).
template <int TY, int TZ, int MINB>
__global__ void __launch_bounds__(32 * TY * TZ, MINB) stage_fp64_blocks_kernel(Grid g, StageArgs a) {
  const int ii = blockIdx.x * 32 + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  stage_point_fp64<32, TY, TZ>(g, a, ii, jj, kk);
}

template <int TY, int TZ, int MINB>
cudaError_t launch_fp64_rows(const Grid& g, const StageArgs& a, cudaStream_t s) {
  if (g.n0 % 32) return cudaErrorInvalidValue;  // the caller checks; rows must be full
  dim3 block(32, TY, TZ);
  dim3 grid(g.n0 / 32, (g.n1 + TY - 1) / TY, (g.n2 + TZ - 1) / TZ);
  if (g.n1 % TY == 0 && g.n2 % TZ == 0 && TY >= 2) {
    constexpr int smem = (int)rows_block_smem(TY, TZ, true);
    if constexpr (smem > 48 * 1024) {  // above the default limit: opt in once per device
      static std::atomic<unsigned> done{0};
      cudaError_t e = smem_optin(stage_fp64_blocks_kernel<TY, TZ, MINB>, smem, done);
      if (e != cudaSuccess) return e;
    }
    stage_fp64_blocks_kernel<TY, TZ, MINB><<<grid, block, smem, s>>>(g, a);
  } else {
    stage_fp64_rows_kernel<TY, TZ, MINB><<<grid, block, 0, s>>>(g, a);
  }
  return cudaGetLastError();
}

template cudaError_t launch_fp64_rows<8, 1, 1>(const Grid&, const StageArgs&, cudaStream_t);
template cudaError_t launch_fp64_rows<4, 1, 1>(const Grid&, const StageArgs&, cudaStream_t);
template cudaError_t launch_fp64_rows<4, 2, 1>(const Grid&, const StageArgs&, cudaStream_t);
template cudaError_t launch_fp64_rows<2, 2, 2>(const Grid&, const StageArgs&, cudaStream_t);

}  // namespace bssn
