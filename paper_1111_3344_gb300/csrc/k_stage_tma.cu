// Mixed-precision fused stage with the heavily differenced fields staged in
// shared memory by the Tensor Memory Accelerator (tile, staged fields and
// accessor: tma_tile.cuh).
//
// Each block owns a tile of TTX x TTY x TTZ interior points.  One thread issues
// one cp.async.bulk.tensor load per staged field -- the field's box over the
// tile plus three ghost layers on every side, cut from the 4-D tensor
// [field][z][y][x] of the float stage buffer -- all completing on one
// mbarrier.  After the wait every thread evaluates the same per-point
// arithmetic as the other stage kernels (rhs_point_acc), reading the staged
// fields from shared memory and the rest through L1.
//
// The wait on the mbarrier is bounded: after WAIT_LIMIT polls the block sets
// the error word (read back by the host as BSSN_ETIMEOUT), waits once more,
// boundedly, for its own copies, and returns without writing results.  A
// test hook (StageArgsT::stall_polls) makes the wait run out on purpose: the
// block then issues no copy at all, polls that many times, sets the error
// word and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tma_tile.cuh"

namespace bssn {

// Sh: tile shape (tma_tile.cuh); MINB: blocks per SM the registers are capped for.
template <typename Sh, int MINB>
__global__ void __launch_bounds__(Sh::TX * Sh::TY * Sh::TZ, MINB)
    stage_mixed_tma_kernel(const __grid_constant__ CUtensorMap tmap, Grid g, StageArgsMixed a,
                           int* __restrict__ err) {
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) unsigned long long mbar;
  // 128-byte aligned start for the TMA destinations
  float* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127) / sizeof(float);
  const int tid = threadIdx.x + Sh::TX * (threadIdx.y + Sh::TY * threadIdx.z);
  const int ii0 = blockIdx.x * Sh::TX, jj0 = blockIdx.y * Sh::TY, kk0 = blockIdx.z * Sh::TZ;
  const unsigned bar = smem_addr(&mbar);
  if (tid == 0) mbar_init(bar);
  __syncthreads();
  const bool stall = a.stall_polls > 0;  // test hook: no copy, short wait
  if (tid == 0 && !stall) issue_staged_loads<Sh>(&tmap, bar, smem, ii0, jj0, kk0);
  if (!mbar_wait(bar, 0, stall ? (long long)a.stall_polls : WAIT_LIMIT)) {
    if (tid == 0) atomicExch(err, 1);
    if (!stall) mbar_wait(bar, 0, WAIT_LIMIT);  // let this block's own copies land before it exits
    return;
  }
  const int ti = threadIdx.x, tj = threadIdx.y, tk = threadIdx.z;
  const int ii = ii0 + ti, jj = jj0 + tj, kk = kk0 + tk;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  const int i = ii + GH, j = jj + GH, k = kk + GH;
  TileAccT<Sh> acc;
  acc.st = a.src;
  acc.id = lin(g, i, j, k);
  acc.fs = g.fstride;
  acc.sd[0] = 1;
  acc.sd[1] = g.pitch;
  acc.sd[2] = g.plane;
  acc.sm = smem + ((tk + GH) * Sh::BY + (tj + GH)) * Sh::BX + (ti + GH);
  stage_point_mixed_acc(g, a, acc, ii, jj, kk);
}

// ------------------------------------------------------------------ host
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}

cudaError_t make_stage_tensor_map(const Grid& g, const float* base, CUtensorMap* out, int variant) {
  // the encoding is a driver call and needs a current context: a thread whose
  // first CUDA call this is has none until a runtime call binds the primary
  // context of its device (cudaFree(nullptr) does, and frees nothing)
  cudaError_t ce = cudaFree(nullptr);
  if (ce != cudaSuccess) return ce;
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&g_encode, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !g_encode) return cudaErrorNotSupported;
  }
  const int by = variant >= 1 ? TmaShape<8>::BY : TmaShape<4>::BY;
  const int bz = TmaShape<4>::BZ;
  cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)g.sy, (cuuint64_t)g.sz, (cuuint64_t)NF};
  cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4, (cuuint64_t)g.fstride * 4};
  cuuint32_t box[4] = {(cuuint32_t)TmaDefault::BX, (cuuint32_t)by, (cuuint32_t)bz, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// dynamic shared memory above the default limit, once per kernel and device
template <typename Sh, int MINB>
static cudaError_t tma_attr() {
  static std::atomic<unsigned> done{0};
  return smem_optin(stage_mixed_tma_kernel<Sh, MINB>, Sh::SMEM, done);
}

template <typename Sh, int MINB>
static cudaError_t launch_tma(const Grid& g, const StageArgsMixed& a, const CUtensorMap& map, int* err,
                              cudaStream_t s) {
  cudaError_t e = tma_attr<Sh, MINB>();
  if (e != cudaSuccess) return e;
  dim3 block(Sh::TX, Sh::TY, Sh::TZ);
  dim3 grid((g.n0 + Sh::TX - 1) / Sh::TX, (g.n1 + Sh::TY - 1) / Sh::TY, (g.n2 + Sh::TZ - 1) / Sh::TZ);
  stage_mixed_tma_kernel<Sh, MINB><<<grid, block, Sh::SMEM, s>>>(map, g, a, err);
  return cudaGetLastError();
}

// variant 0: 32 x 4 x 1 tiles, two blocks per SM; 1: 32 x 8 x 1 tiles, one
// block per SM (half the shared memory per SM, so more L1 for the fields read
// through it); 2: 32 x 8 x 1 tiles staging beta^i as well (eleven fields,
// 173 KB, one block per SM; the tensor map of variant 1 serves, same box);
// map: a tensor map made for the same variant
cudaError_t prepare_stage_mixed_tma(int variant) {
  if (variant == 2) return tma_attr<TmaShape<8, 1, 11>, 1>();
  return variant == 1 ? tma_attr<TmaShape<8>, 1>() : tma_attr<TmaShape<4>, 2>();
}

cudaError_t launch_stage_mixed_tma(const Grid& g, const StageArgsMixed& a, const CUtensorMap& map,
                                   int* err, cudaStream_t s, int variant) {
  if (variant == 2) return launch_tma<TmaShape<8, 1, 11>, 1>(g, a, map, err, s);
  return variant == 1 ? launch_tma<TmaShape<8>, 1>(g, a, map, err, s) : launch_tma<TmaShape<4>, 2>(g, a, map, err, s);
}

}  // namespace bssn
