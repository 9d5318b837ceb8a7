// Batched evolutions in double-word precision (BSSN_FF): one block per tile
// of one work list, as the one-block-per-tile float64 kernels of k_batch.cu,
// each thread running the double-word stage of the single-grid kernels
// (stage_point_ff) -- so a member's result is the same alone, in the mix, or
// through a bssn_ctx with a full-row configuration of the same register cap.
// FULL: every member of the list has full tiles (n0 a multiple of 32, n1 of
// TY, n2 of TZ), so warps share first differences across lanes and rows share
// them through shared memory; the others run the every-stencil form.  The
// boundary launch covers every member's ghost points (Sommerfeld in
// double-word arithmetic, or periodic copies).
#include <cuda_runtime.h>

#include "batch_internal.cuh"
#include "boundary_point.cuh"
#include "stage_point.cuh"

namespace bssn {

__device__ __forceinline__ int find_member_ff(const unsigned* base, int count, unsigned t) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int TY, int TZ, int MINB, bool FULL>
__global__ void __launch_bounds__(32 * TY * TZ, MINB)
    batch_tile_ff_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk, int stage) {
  __shared__ int sid;
  __shared__ unsigned slocal;
  const int tid = threadIdx.x + 32 * (threadIdx.y + TY * threadIdx.z);
  const unsigned t = blockIdx.x;
  if (t >= wk->total_tiles) return;  // whole block
  if (tid == 0) {
    const int slot = find_member_ff(wk->tile_base, wk->count, t);
    sid = wk->member[slot];
    slocal = t - wk->tile_base[slot];
  }
  __syncthreads();
  const MemberDev& M = mem[sid];
  unsigned lt = slocal;
  const int bx = (int)(lt % (unsigned)M.tiles[0]);
  lt /= (unsigned)M.tiles[0];
  const int by = (int)(lt % (unsigned)M.tiles[1]);
  const int bz = (int)(lt / (unsigned)M.tiles[1]);
  const int ii = bx * 32 + threadIdx.x, jj = by * TY + threadIdx.y, kk = bz * TZ + threadIdx.z;
  if constexpr (FULL) {
    stage_point_ff<32, TY, TZ>(M.g, M.aff[stage], ii, jj, kk);  // every thread inside the grid
  } else {
    if (ii < M.g.n0 && jj < M.g.n1 && kk < M.g.n2) stage_point_ff<0>(M.g, M.aff[stage], ii, jj, kk);
  }
}

__global__ void batch_boundary_ff_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk,
                                         int stage) {
  const unsigned long long total = wk->total_bc;
  const int count = wk->count;
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (wk->bc_base[mid] <= t) lo = mid;
      else hi = mid;
    }
    const MemberDev& M = mem[wk->member[lo]];
    const unsigned q = (unsigned)(t - wk->bc_base[lo]);
    const StageArgsFF& a = M.aff[stage];
    if (M.g.periodic) {
      // the copy moves 8-byte values whatever they hold
      periodic_point<double>(M.g, reinterpret_cast<double*>(a.out0), nullptr, q);
      if (a.mode == MODE_LAST) periodic_point<double>(M.g, a.yn, nullptr, q);
    } else {
      sommerfeld_point_ff(M.g, a, a.kshell, q);
    }
  }
}

// configurations: 32 x TY x TZ tiles, registers capped for MINB blocks per SM
struct FfBatchCfg {
  const char* name;
  int ty, tz;
  const void* kfull;
  const void* krest;
};
#define FCFG(TY, TZ, MINB)                                                  \
  { "fftiles32x" #TY "x" #TZ "/" #MINB, TY, TZ,                            \
    (const void*)batch_tile_ff_kernel<TY, TZ, MINB, true>,                 \
    (const void*)batch_tile_ff_kernel<TY, TZ, MINB, false> }
static const FfBatchCfg k_ffcfg[] = {FCFG(4, 1, 8), FCFG(4, 1, 4)};
#undef FCFG

int batch_ff_config_count() { return (int)(sizeof(k_ffcfg) / sizeof(k_ffcfg[0])); }
const char* batch_ff_config_name(int v) { return k_ffcfg[v].name; }
void batch_ff_tile_shape(int v, int& tx, int& ty, int& tz) {
  tx = 32;
  ty = k_ffcfg[v].ty;
  tz = k_ffcfg[v].tz;
}

cudaError_t launch_batch_stage_ff(int v, bool full, const MemberDev* mem, const BatchWork* wk, unsigned ntiles,
                                  int stage, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  const FfBatchCfg& c = k_ffcfg[v];
  const void* fn = full ? c.kfull : c.krest;
  const size_t smem = full ? (size_t)11 * (c.ty + 4) * c.tz * 32 * sizeof(ff) : 0;
  void* args[] = {(void*)&mem, (void*)&wk, (void*)&stage};
  return cudaLaunchKernel(fn, dim3(ntiles), dim3(32, c.ty, c.tz), args, smem, s);
}

cudaError_t launch_batch_boundary_ff(const MemberDev* mem, const BatchWork* wk, int stage, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  batch_boundary_ff_kernel<<<sms * 8, 128, 0, s>>>(mem, wk, stage);
  return cudaGetLastError();
}

}  // namespace bssn
