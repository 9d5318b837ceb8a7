// Double-word fused stage kernels for blocks whose warps are full rows of 32
// x points (n0 a multiple of 32): the mixed second differences D1_x D1_y and
// D1_x D1_z take the neighbouring points' first differences from the
// neighbouring lanes and, when n1 and n2 fill the blocks, D1_y D1_z takes the
// neighbouring rows' from shared memory -- the float64 path's arrangement
// (k_stage_shfl.cu) in double-word arithmetic.  Instantiated for several
// register caps in k_stage_ff_rows.cu and k_stage_ff_rows_occ.cu (compiled in
// parallel).
#pragma once
#include "stage_point.cuh"

namespace bssn {

cudaError_t launch_ff_any(const Grid& g, const StageArgsFF& a, cudaStream_t s);

// warps of full 32-point rows (n0 a multiple of 32); whole warps leave together
template <int TY, int TZ, int MINB>
__global__ void __launch_bounds__(32 * TY * TZ, MINB) stage_ff_rows_kernel(Grid g, StageArgsFF a) {
  const int ii = blockIdx.x * 32 + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  if (jj >= g.n1 || kk >= g.n2) return;
  stage_point_ff<32>(g, a, ii, jj, kk);
}
// full blocks (n1 % TY == 0, n2 % TZ == 0 as well): D_y D_z through shared memory
template <int TY, int TZ, int MINB>
__global__ void __launch_bounds__(32 * TY * TZ, MINB) stage_ff_blocks_kernel(Grid g, StageArgsFF a) {
  const int ii = blockIdx.x * 32 + threadIdx.x;
  const int jj = blockIdx.y * TY + threadIdx.y;
  const int kk = blockIdx.z * TZ + threadIdx.z;
  stage_point_ff<32, TY, TZ>(g, a, ii, jj, kk);
}

// 32-wide rows when n0 is a multiple of 32 (full blocks when n1, n2 fill
// them too), else the every-stencil kernel of the same block shape
template <int TY, int TZ, int MINB>
cudaError_t launch_ff_rows(const Grid& g, const StageArgsFF& a, cudaStream_t s) {
  if (g.n0 % 32) return launch_ff_any(g, a, s);
  dim3 block(32, TY, TZ);
  dim3 grid(g.n0 / 32, (g.n1 + TY - 1) / TY, (g.n2 + TZ - 1) / TZ);
  if (g.n1 % TY == 0 && g.n2 % TZ == 0 && TY >= 2) {
    constexpr int smem = (int)rows_block_smem(TY, TZ, false);
    if constexpr (smem > 48 * 1024) {  // above the default limit: opt in once per device
      static std::atomic<unsigned> done{0};
      cudaError_t e = smem_optin(stage_ff_blocks_kernel<TY, TZ, MINB>, smem, done);
      if (e != cudaSuccess) return e;
    }
    stage_ff_blocks_kernel<TY, TZ, MINB><<<grid, block, smem, s>>>(g, a);
  } else {
    stage_ff_rows_kernel<TY, TZ, MINB><<<grid, block, 0, s>>>(g, a);
  }
  return cudaGetLastError();
}

}  // namespace bssn
