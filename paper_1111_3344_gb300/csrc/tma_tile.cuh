// Shared-memory tile of the TMA-staged mixed stage kernels (single grid:
// k_stage_tma.cu; batched: k_batch_tma.cu): tile shape, the staged fields,
// the accessor that reads them from shared memory, and the bounded mbarrier
// wait.
//
// A block owns TTX x TTY x TTZ interior points.  One cp.async.bulk.tensor load
// per staged field brings the field's box over the tile plus three ghost
// layers on every side (BXP x BYP x BZP floats; BXP rounded up so that a box
// row is a multiple of 16 bytes).  The staged fields are the eight with second
// derivatives and the widest stencils, W, the six gt_ij and alpha, and in the
// eleven-field form also the three beta^i (second-differenced as well).
#pragma once
#include <cuda.h>

#include "stage_point.cuh"

namespace bssn {

constexpr int NSTAGED = 8;
constexpr long long WAIT_LIMIT = 1LL << 24;

// Tile of 32 x TY x TZ interior points and its boxes: BX = 32 + 6 rounded up
// to a multiple of 4 floats, BY = TY + 6, BZ = TZ + 6 (three ghost layers on
// every side); slots of the staged fields 128-byte aligned.  NST: staged
// fields, 8 (W, gt_ij, alpha) or 11 (and beta^i).
template <int TY_, int TZ_ = 1, int NST_ = NSTAGED>
struct TmaShape {
  static constexpr int TX = 32, TY = TY_, TZ = TZ_, NST = NST_;
  static constexpr int BX = 40, BY = TY + 2 * GH, BZ = TZ + 2 * GH;
  static constexpr int BOX = BX * BY * BZ;                              // floats of one field's box
  static constexpr int SLOT = (BOX + 31) / 32 * 32;                     // slot stride
  static constexpr unsigned BYTES = NST * BOX * sizeof(float);         // bytes the copies deliver
  static constexpr int SMEM = NST * SLOT * (int)sizeof(float) + 128;  // + alignment slack
};

// the 32 x 4 x 1 tile (two blocks per SM): the batched kernel and the names below
using TmaDefault = TmaShape<4>;
constexpr int TTX = TmaDefault::TX, TTY = TmaDefault::TY, TTZ = TmaDefault::TZ;
constexpr int BXP = TmaDefault::BX, BYP = TmaDefault::BY, BZP = TmaDefault::BZ;
constexpr int BOXF = TmaDefault::BOX, SLOTF = TmaDefault::SLOT;
constexpr unsigned STAGED_BYTES = TmaDefault::BYTES;
constexpr int SMEM_BYTES = TmaDefault::SMEM;

// slot s -> field: W, gt_ij (6), alpha, then beta^i (slots 8-10, staged when
// the shape has NST = 11)
__host__ __device__ __forceinline__ int staged_field(int s) {
  return s == 0 ? F_CHI : (s <= 6 ? F_GT + (s - 1) : (s == 7 ? F_ALP : F_BETA + (s - 8)));
}
// field -> slot, -1 for a field read through L1
template <int NST = NSTAGED>
__device__ __forceinline__ int staged_slot(int f) {
  if (f == F_CHI) return 0;
  if (f >= F_GT && f < F_GT + 6) return 1 + (f - F_GT);
  if (f == F_ALP) return 7;
  if (NST > 8 && f >= F_BETA && f < F_BETA + 3) return 8 + (f - F_BETA);
  return -1;
}

// Accessor: staged fields from the shared box, the others from global.
template <typename Sh>
struct TileAccT {
  const float* __restrict__ st;
  long long id, fs, sd[3];
  const float* sm;  // shared address of this point in slot 0
  __device__ __forceinline__ const float* ptr(int f) const {
    const int sl = staged_slot<Sh::NST>(f);
    return sl >= 0 ? sm + sl * Sh::SLOT : st + (long long)f * fs + id;
  }
  __device__ __forceinline__ long long s(int f, int d) const {
    return staged_slot<Sh::NST>(f) >= 0 ? (d == 0 ? 1 : (d == 1 ? Sh::BX : Sh::BX * Sh::BY)) : sd[d];
  }
  template <typename T>
  __device__ __forceinline__ T ld(int f, const float* p) const {
    return staged_slot<Sh::NST>(f) >= 0 ? T(*p) : T(__ldg(p));
  }
};
using TileAcc = TileAccT<TmaDefault>;

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

__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Thread 0: arm the barrier for the staged bytes and issue one tensor load per
// staged field, box origin (x0, y0, z0) in stored coordinates (the interior
// start of the tile minus the ghost width; x0 a multiple of 32, so the
// innermost offset is a multiple of 16 bytes).  The tensor map's box is
// Sh::BX x Sh::BY x Sh::BZ.
template <typename Sh = TmaDefault>
__device__ __forceinline__ void issue_staged_loads(const void* tmap, unsigned bar, float* smem, int x0, int y0,
                                                   int z0) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(Sh::BYTES)
               : "memory");
#pragma unroll
  for (int s = 0; s < Sh::NST; s++) {
    const int f = staged_field(s);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(smem + s * Sh::SLOT)),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x0), "r"(y0), "r"(z0), "r"(f), "r"(bar)
        : "memory");
  }
}

}  // namespace bssn
