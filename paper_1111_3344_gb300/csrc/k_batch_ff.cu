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
  // the member's grid and stage arguments are copied to shared memory once per
  // block: under a tight register cap the point function reloads them often,
  // and shared loads are cheaper than loads of the member table
  __shared__ Grid sg;
  __shared__ StageArgsFF sa;
  __shared__ int stile[2];
  __shared__ unsigned slocal;
  const int tid = threadIdx.x + 32 * (threadIdx.y + TY * threadIdx.z);
  const unsigned t = blockIdx.x;
  if (t >= wk->total_tiles) return;  // whole block
  if (tid == 0) {
    const int slot = find_member_ff(wk->tile_base, wk->count, t);
    const MemberDev& M = mem[wk->member[slot]];
    sg = M.g;
    sa = M.aff[stage];
    stile[0] = M.tiles[0];
    stile[1] = M.tiles[1];
    slocal = t - wk->tile_base[slot];
  }
  __syncthreads();
  unsigned lt = slocal;
  const int bx = (int)(lt % (unsigned)stile[0]);
  lt /= (unsigned)stile[0];
  const int by = (int)(lt % (unsigned)stile[1]);
  const int bz = (int)(lt / (unsigned)stile[1]);
  const int ii = bx * 32 + threadIdx.x, jj = by * TY + threadIdx.y, kk = bz * TZ + threadIdx.z;
  if constexpr (FULL) {
    stage_point_ff<32, TY, TZ>(sg, sa, ii, jj, kk);  // every thread inside the grid
  } else {
    if (ii < sg.n0 && jj < sg.n1 && kk < sg.n2) stage_point_ff<0>(sg, sa, ii, jj, kk);
  }
}

__global__ void batch_boundary_ff_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk,
                                         int stage) {
  __shared__ BcList L;
  const unsigned long long total = wk->total_bc;
  const int count = wk->count;
  load_bc_list(L, wk, count);
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int lo = find_bc(L, count, t);
    const MemberDev& M = mem[L.member[lo]];
    const unsigned q = (unsigned)(t - L.base[lo]);
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

// configurations: 32 x TY x TZ tiles, registers capped for MF blocks per SM
// in the full-tile kernel and MR in the every-stencil one (which spills more
// at the same cap)
struct FfBatchCfg {
  const char* name;
  int ty, tz;
  const void* kfull;
  const void* krest;
};
#define FCFG(TY, TZ, MF, MR)                                                \
  { "fftiles32x" #TY "x" #TZ "/" #MF "+" #MR, TY, TZ,                      \
    (const void*)batch_tile_ff_kernel<TY, TZ, MF, true>,                   \
    (const void*)batch_tile_ff_kernel<TY, TZ, MR, false> }
static const FfBatchCfg k_ffcfg[] = {FCFG(4, 1, 8, 4), FCFG(4, 1, 8, 8), FCFG(4, 1, 4, 4)};
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
  const size_t smem = full ? rows_block_smem(c.ty, c.tz, false) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
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
