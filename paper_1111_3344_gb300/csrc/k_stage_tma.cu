// Mixed-precision fused stage with the heavily differenced fields staged in
// shared memory by the Tensor Memory Accelerator.
//
// Each block owns a tile of TX x TY x TZ interior points.  One thread issues
// one cp.async.bulk.tensor load per staged field -- the field's box over the
// tile plus three ghost layers on every side, cut from the 4-D tensor
// [field][z][y][x] of the float stage buffer -- all completing on one
// mbarrier.  The staged fields are the eight with second derivatives and the
// widest stencils: W, the six gt_ij and alpha (about half of all stencil
// reads of a point).  After the wait every thread evaluates the same
// per-point arithmetic as the other stage kernels (rhs_point_acc), reading
// the staged fields from shared memory and the rest through L1.
//
// The wait on the mbarrier is bounded: after WAIT_LIMIT polls the block sets
// the error word (read back by the host as BSSN_ETIMEOUT), waits once more,
// boundedly, for its own copies, and returns without writing results.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "stage_point.cuh"

namespace bssn {

constexpr int TTX = 32, TTY = 4, TTZ = 1;
constexpr int BXP = 40;            // box extent in x: TTX + 6 rounded up to a multiple of 4 floats
constexpr int BYP = TTY + 2 * GH;  // 10
constexpr int BZP = TTZ + 2 * GH;  // 7
constexpr int BOXF = BXP * BYP * BZP;             // floats of one field's box (2800)
constexpr int SLOTF = (BOXF + 31) / 32 * 32;      // slot stride: 128-byte aligned boxes
constexpr int NSTAGED = 8;
constexpr unsigned STAGED_BYTES = NSTAGED * BOXF * sizeof(float);  // bytes the copies deliver
constexpr int SMEM_BYTES = NSTAGED * SLOTF * (int)sizeof(float) + 128;  // + alignment slack
constexpr long long WAIT_LIMIT = 1LL << 24;

__host__ __device__ __forceinline__ int staged_field(int s) {
  return s == 0 ? F_CHI : (s <= 6 ? F_GT + (s - 1) : F_ALP);
}
__device__ __forceinline__ int staged_slot(int f) {
  return f == F_CHI ? 0 : ((f >= F_GT && f < F_GT + 6) ? 1 + (f - F_GT) : (f == F_ALP ? 7 : -1));
}

// Accessor: staged fields from the shared box, the others from global.
struct TileAcc {
  const float* __restrict__ st;
  long long id, fs, sd[3];
  const float* sm;  // shared address of this point in slot 0
  __device__ __forceinline__ const float* ptr(int f) const {
    const int sl = staged_slot(f);
    return sl >= 0 ? sm + sl * SLOTF : st + (long long)f * fs + id;
  }
  __device__ __forceinline__ long long s(int f, int d) const {
    return staged_slot(f) >= 0 ? (d == 0 ? 1 : (d == 1 ? BXP : BXP * BYP)) : sd[d];
  }
  template <typename T>
  __device__ __forceinline__ T ld(int f, const float* p) const {
    return staged_slot(f) >= 0 ? T(*p) : T(__ldg(p));
  }
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit) {
  for (long long it = 0; it < limit; it++) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(TTX * TTY * TTZ, 2)
    stage_mixed_tma_kernel(const __grid_constant__ CUtensorMap tmap, Grid g, StageArgsMixed a,
                           int* __restrict__ err) {
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) unsigned long long mbar;
  // 128-byte aligned start for the TMA destinations
  float* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127) / sizeof(float);
  const int tid = threadIdx.x + TTX * (threadIdx.y + TTY * threadIdx.z);
  const int ii0 = blockIdx.x * TTX, jj0 = blockIdx.y * TTY, kk0 = blockIdx.z * TTZ;
  const unsigned bar = smem_addr(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(STAGED_BYTES)
                 : "memory");
    // box origin in stored coordinates: interior start minus the ghost width
    const int x0 = ii0, y0 = jj0, z0 = kk0;
#pragma unroll
    for (int s = 0; s < NSTAGED; s++) {
      const int f = staged_field(s);
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(smem + s * SLOTF)),
          "l"(reinterpret_cast<unsigned long long>(&tmap)), "r"(x0), "r"(y0), "r"(z0), "r"(f), "r"(bar)
          : "memory");
    }
  }
  if (!mbar_wait(bar, 0, WAIT_LIMIT)) {
    if (tid == 0) atomicExch(err, 1);
    mbar_wait(bar, 0, WAIT_LIMIT);  // let this block's own copies land before it exits
    return;
  }
  const int ti = threadIdx.x, tj = threadIdx.y, tk = threadIdx.z;
  const int ii = ii0 + ti, jj = jj0 + tj, kk = kk0 + tk;
  if (ii >= g.n0 || jj >= g.n1 || kk >= g.n2) return;
  const int i = ii + GH, j = jj + GH, k = kk + GH;
  TileAcc acc;
  acc.st = a.src;
  acc.id = lin(g, i, j, k);
  acc.fs = g.fstride;
  acc.sd[0] = 1;
  acc.sd[1] = g.pitch;
  acc.sd[2] = g.plane;
  acc.sm = smem + ((tk + GH) * BYP + (tj + GH)) * BXP + (ti + GH);
  stage_point_mixed_acc(g, a, acc, ii, jj, kk);
}

// ------------------------------------------------------------------ host
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}

cudaError_t make_stage_tensor_map(const Grid& g, const float* base, CUtensorMap* out) {
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&g_encode, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !g_encode) return cudaErrorNotSupported;
  }
  cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)g.sy, (cuuint64_t)g.sz, (cuuint64_t)NF};
  cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4, (cuuint64_t)g.fstride * 4};
  cuuint32_t box[4] = {BXP, BYP, BZP, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_stage_mixed_tma(const Grid& g, const StageArgsMixed& a, const CUtensorMap& map,
                                   int* err, cudaStream_t s) {
  static bool attr = false;
  const int bytes = SMEM_BYTES;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(stage_mixed_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 block(TTX, TTY, TTZ);
  dim3 grid((g.n0 + TTX - 1) / TTX, (g.n1 + TTY - 1) / TTY, (g.n2 + TTZ - 1) / TTZ);
  stage_mixed_tma_kernel<<<grid, block, bytes, s>>>(map, g, a, err);
  return cudaGetLastError();
}

}  // namespace bssn
