// Batched mixed-precision stage with the heavily differenced fields staged in
// shared memory by the Tensor Memory Accelerator: the persistent form of
// stage_mixed_tma_kernel (k_stage_tma.cu) over every active member's tiles.
//
// Each block takes tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... of the
// batch's work list.  Per tile, thread 0 reads the member's arguments into
// shared memory, then issues the tensor loads of the tile's boxes (one per
// staged field: 8 on 32x4x1 tiles, or 11 with beta^i on 32x8x1 tiles) with
// the member's tensor map for this stage (held in the member table in device
// memory, written by the host before the launch), all completing on one
// mbarrier whose phase alternates from tile to tile.  Every thread then
// evaluates the same per-point stage as the single-grid kernel.
//
// The wait on the mbarrier is bounded.  Whether the block gives up is decided
// for the whole block at once (a barrier vote), so that no thread leaves while
// others wait at a barrier: on a timeout the block sets the error word, waits
// once more, boundedly, for its own copies, and returns.  With the test hook
// StageArgsT::stall_polls set in the member's arguments the block issues no
// copy and gives up after that many polls.
#include "batch_internal.cuh"
#include "tma_tile.cuh"

namespace bssn {

namespace {

__device__ __forceinline__ int find_member_tma(const unsigned* __restrict__ base, int count, unsigned t) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <typename Sh, int MINB>
__global__ void __launch_bounds__(Sh::TX * Sh::TY * Sh::TZ, MINB)
    batch_stage_tma_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk, int stage,
                           int* __restrict__ err) {
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ Grid sg;
  __shared__ StageArgsMixed sa;
  __shared__ int stile[2];
  __shared__ unsigned slocal;
  __shared__ const CUtensorMap* smap;
  float* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127) / sizeof(float);
  const int tid = threadIdx.x + Sh::TX * (threadIdx.y + Sh::TY * threadIdx.z);
  const unsigned bar = smem_addr(&mbar);
  if (tid == 0) mbar_init(bar);
  const unsigned total = wk->total_tiles;
  const int count = wk->count;
  unsigned phase = 0;
  // thread 0: tile range [t_lo, t_hi) of the member whose arguments are in
  // shared memory (a block's next tile, gridDim.x further on, is nearly
  // always in the same member: no search and no copy then)
  unsigned t_lo = 1u, t_hi = 0u;
  for (unsigned t = blockIdx.x; t < total; t += gridDim.x) {
    // the previous tile is done with the shared arguments and the boxes
    __syncthreads();
    if (tid == 0) {
      if (t < t_lo || t >= t_hi) {
        const int slot = find_member_tma(wk->tile_base, count, t);
        const MemberDev& M = mem[wk->member[slot]];
        sg = M.g;
        sa = M.amx[stage];
        stile[0] = M.tiles[0];
        stile[1] = M.tiles[1];
        smap = &M.tmap[stage];
        t_lo = wk->tile_base[slot];
        t_hi = wk->tile_base[slot + 1];
      }
      slocal = t - t_lo;
    }
    __syncthreads();
    unsigned lt = slocal;
    const int bx = (int)(lt % (unsigned)stile[0]);
    lt /= (unsigned)stile[0];
    const int by = (int)(lt % (unsigned)stile[1]);
    const int bz = (int)(lt / (unsigned)stile[1]);
    const int ii0 = bx * Sh::TX, jj0 = by * Sh::TY, kk0 = bz * Sh::TZ;
    const bool stall = sa.stall_polls > 0;  // test hook: no copy, short wait
    if (tid == 0) {
      // the map was written through the generic proxy (a copy from the host)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(smap) : "memory");
      // the boxes were last read through the generic proxy; the loads write them
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (!stall) issue_staged_loads<Sh>(smap, bar, smem, ii0, jj0, kk0);
    }
    const bool ok = mbar_wait(bar, phase, stall ? (long long)sa.stall_polls : WAIT_LIMIT);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(err, 1);
        if (!stall) mbar_wait(bar, phase, WAIT_LIMIT);  // let this block's own copies land before it exits
      }
      return;
    }
    phase ^= 1u;
    const int ti = threadIdx.x, tj = threadIdx.y, tk = threadIdx.z;
    const int ii = ii0 + ti, jj = jj0 + tj, kk = kk0 + tk;
    if (ii < sg.n0 && jj < sg.n1 && kk < sg.n2) {
      const int i = ii + GH, j = jj + GH, k = kk + GH;
      TileAccT<Sh> acc;
      acc.st = sa.src;
      acc.id = lin(sg, i, j, k);
      acc.fs = sg.fstride;
      acc.sd[0] = 1;
      acc.sd[1] = sg.pitch;
      acc.sd[2] = sg.plane;
      acc.sm = smem + ((tk + GH) * Sh::BY + (tj + GH)) * Sh::BX + (ti + GH);
      stage_point_mixed_acc(sg, sa, acc, ii, jj, kk);
    }
  }
}

}  // namespace

// variant 0: 32x4x1 tiles, 8 staged fields, two blocks per SM; 1: 32x8x1
// tiles, 11 staged fields (beta^i too), one block per SM
using BatchTma0 = TmaShape<4>;
using BatchTma1 = TmaShape<8, 1, 11>;

void batch_tma_tile_shape(int v, int& tx, int& ty, int& tz) {
  tx = 32;
  ty = v == 1 ? BatchTma1::TY : BatchTma0::TY;
  tz = 1;
}

// Dynamic shared memory above the default limit; called when the batch
// selects this kernel, outside graph capture.
cudaError_t prepare_batch_stage_tma(int v) {
  if (v == 1)
    return cudaFuncSetAttribute(batch_stage_tma_kernel<BatchTma1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                BatchTma1::SMEM);
  return cudaFuncSetAttribute(batch_stage_tma_kernel<BatchTma0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              BatchTma0::SMEM);
}

template <typename Sh, int MINB>
static cudaError_t launch_tma_b(const MemberDev* mem, const BatchWork* wk, int stage, int* err, cudaStream_t s) {
  const int bytes = Sh::SMEM;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_stage_tma_kernel<Sh, MINB>,
                                                      Sh::TX * Sh::TY * Sh::TZ, bytes);
  if (e != cudaSuccess) return e;
  if (per < 1) per = 1;
  batch_stage_tma_kernel<Sh, MINB><<<sms * per, dim3(Sh::TX, Sh::TY, Sh::TZ), bytes, s>>>(mem, wk, stage, err);
  return cudaGetLastError();
}

cudaError_t launch_batch_stage_tma(int v, const MemberDev* mem, const BatchWork* wk, int stage, int* err,
                                   cudaStream_t s) {
  return v == 1 ? launch_tma_b<BatchTma1, 1>(mem, wk, stage, err, s)
                : launch_tma_b<BatchTma0, 2>(mem, wk, stage, err, s);
}

}  // namespace bssn
