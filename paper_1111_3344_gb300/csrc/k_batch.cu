// Batched evolutions: one persistent launch per RK4 stage over the tiles of
// every active member, and one launch for all their boundaries.
//
// Blocks stride over the global tile index; a tile's member is found by binary
// search in the work-list prefix sums, its grid and stage arguments are staged
// in shared memory, and each thread runs the same per-point stage function as
// the single-grid kernels (stage_point.cuh) -- so a member's result does not
// depend on which other members share the launch, or on the tile shape.
#include <cuda_runtime.h>

#include "batch_internal.cuh"
#include "boundary_point.cuh"
#include "stage_point.cuh"

namespace bssn {

__device__ __forceinline__ int find_member(const unsigned* base, int count, unsigned t) {
  int lo = 0, hi = count;  // largest lo with base[lo] <= t
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int TX, int TY, int TZ, int MINB>
__global__ void __launch_bounds__(TX * TY * TZ, MINB)
    batch_stage_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk, int stage) {
  __shared__ Grid sg;
  __shared__ StageArgsMixed sa;
  __shared__ int stile[3];
  __shared__ unsigned slocal;
  const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
  const unsigned total = wk->total_tiles;
  const int count = wk->count;
  // thread 0: tile range [t_lo, t_hi) of the member whose arguments are in
  // shared memory (a block's next tile, gridDim.x further on, is nearly
  // always in the same member: no search and no copy then)
  unsigned t_lo = 1u, t_hi = 0u;
  for (unsigned t = blockIdx.x; t < total; t += gridDim.x) {
    __syncthreads();  // the previous tile is done with the shared arguments
    if (tid == 0) {
      if (t < t_lo || t >= t_hi) {
        const int slot = find_member(wk->tile_base, count, t);
        const MemberDev& M = mem[wk->member[slot]];
        sg = M.g;
        sa = M.amx[stage];
        stile[0] = M.tiles[0];
        stile[1] = M.tiles[1];
        stile[2] = M.tiles[2];
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
    const int ii = bx * TX + threadIdx.x, jj = by * TY + threadIdx.y, kk = bz * TZ + threadIdx.z;
    if (ii < sg.n0 && jj < sg.n1 && kk < sg.n2) stage_point_mixed(sg, sa, ii, jj, kk);
  }
}

// Float64 persistent stage: the body of one tile is a call of its own
// (__noinline__), so that it gets the register allocation of a one-tile
// kernel.  Inlined into the loop over tiles, the float64 stage spills
// 1.2-1.8 KB per thread whether its arguments sit in shared memory or in the
// member table; behind the call, about 330 B (full tiles, 255 registers).  The callee reads the member's grid and
// stage arguments from the read-only member table.  FULL: the member has full
// tiles (every warp a full x-row, every thread of the block inside the grid),
// which the caller decides uniformly over the block.
template <int TY, int TZ, bool FULL>
__device__ __noinline__ void batch_fp64_tile(const MemberDev* __restrict__ mem, int sid, unsigned lt, int stage) {
  const MemberDev& M = mem[sid];
  const int bx = (int)(lt % (unsigned)M.tiles[0]);
  lt /= (unsigned)M.tiles[0];
  const int by = (int)(lt % (unsigned)M.tiles[1]);
  const int bz = (int)(lt / (unsigned)M.tiles[1]);
  const int ii = bx * 32 + threadIdx.x, jj = by * TY + threadIdx.y, kk = bz * TZ + threadIdx.z;
  if constexpr (FULL)
    stage_point_fp64<32, TY, TZ>(M.g, M.a64[stage], ii, jj, kk);
  else if (ii < M.g.n0 && jj < M.g.n1 && kk < M.g.n2)
    stage_point_fp64<0>(M.g, M.a64[stage], ii, jj, kk);
}

template <int TY, int TZ, int MINB>
__global__ void __launch_bounds__(32 * TY * TZ, MINB)
    batch_stage_fp64_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk, int stage) {
  __shared__ int sid, sfull;
  __shared__ unsigned slocal;
  const int tid = threadIdx.x + 32 * (threadIdx.y + TY * threadIdx.z);
  const unsigned total = wk->total_tiles;
  const int count = wk->count;
  // thread 0: the member of the block's current tile and its tile range
  unsigned t_lo = 1u, t_hi = 0u;
  int cur = 0, full = 0;
  for (unsigned t = blockIdx.x; t < total; t += gridDim.x) {
    __syncthreads();  // the previous tile is done with sid, sfull, slocal
    if (tid == 0) {
      if (t < t_lo || t >= t_hi) {
        const int slot = find_member(wk->tile_base, count, t);
        cur = wk->member[slot];
        const Grid& g = mem[cur].g;
        full = g.n0 % 32 == 0 && g.n1 % TY == 0 && g.n2 % TZ == 0;
        t_lo = wk->tile_base[slot];
        t_hi = wk->tile_base[slot + 1];
      }
      sid = cur;
      sfull = full;
      slocal = t - t_lo;
    }
    __syncthreads();
    if (sfull) batch_fp64_tile<TY, TZ, true>(mem, sid, slocal, stage);
    else batch_fp64_tile<TY, TZ, false>(mem, sid, slocal, stage);
  }
}

// One block per tile of one work list (grid = the list's tile count): the
// block looks up its member once and runs one point function.  Against the
// persistent kernel above this trades the resident-block loop for a launch
// over all tiles; the compiler then allocates registers as for a single-grid
// stage (about 200 B of spills per thread for float64, against 1.2-1.8 KB in
// the loop).  FULL (float64): every member of the list has full tiles, so every
// warp is a full x-row and every thread of a block is inside the grid.
template <int TX, int TY, int TZ, int MINB, bool MIXED, bool FULL>
__global__ void __launch_bounds__(TX * TY * TZ, MINB)
    batch_tile_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk, int stage) {
  __shared__ int sid;
  __shared__ unsigned slocal;
  const int tid = threadIdx.x + TX * (threadIdx.y + TY * threadIdx.z);
  const unsigned t = blockIdx.x;
  if (t >= wk->total_tiles) return;  // whole block
  if (tid == 0) {
    const int slot = find_member(wk->tile_base, wk->count, t);
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
  const int ii = bx * TX + threadIdx.x, jj = by * TY + threadIdx.y, kk = bz * TZ + threadIdx.z;
  if (ii < M.g.n0 && jj < M.g.n1 && kk < M.g.n2) {
    if constexpr (MIXED)
      stage_point_mixed(M.g, M.amx[stage], ii, jj, kk);
    else if constexpr (FULL && TX == 32)
      stage_point_fp64<32, TY, TZ>(M.g, M.a64[stage], ii, jj, kk);
    else
      stage_point_fp64<0>(M.g, M.a64[stage], ii, jj, kk);
  }
}

template <bool MIXED>
__global__ void batch_boundary_kernel(const MemberDev* __restrict__ mem, const BatchWork* __restrict__ wk,
                                      int stage) {
  __shared__ BcList L;
  const unsigned long long total = wk->total_bc;
  const int count = wk->count;
  load_bc_list(L, wk, count);
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int slot = find_bc(L, count, t);
    const MemberDev& M = mem[L.member[slot]];
    const unsigned long long local = t - L.base[slot];
    if (M.g.periodic) {
      const unsigned q = (unsigned)local;
      if constexpr (MIXED) {
        if (blockIdx.y != 0) continue;  // the first field group copies every field
        const StageArgsMixed& a = M.amx[stage];
        periodic_point<float>(M.g, a.out0, a.out0w, q);
        if (a.mode == MODE_LAST) periodic_point<double>(M.g, a.yn, nullptr, q);
      } else {
        const StageArgs& a = M.a64[stage];
        periodic_point<double>(M.g, a.mode == MODE_LAST ? a.yn : a.out0, nullptr, q);
      }
    } else if constexpr (MIXED) {
      // blockIdx.y: one of four field groups (as sommerfeld_mixed_kernel)
      const StageArgsMixed& a = M.amx[stage];
      const unsigned q = (unsigned)local;
      switch (blockIdx.y) {
        case 0: sommerfeld_point_mixed_fields<0, 7, true>(M.g, a, a.kshell, q); break;
        case 1: sommerfeld_point_mixed_fields<7, 13, true>(M.g, a, a.kshell, q); break;
        case 2: sommerfeld_point_mixed_fields<13, 18, true>(M.g, a, a.kshell, q); break;
        default: sommerfeld_point_mixed_fields<18, NF, true>(M.g, a, a.kshell, q); break;
      }
    } else {
      const StageArgs& a = M.a64[stage];
      sommerfeld_point_fp64(M.g, a, a.kshell, (unsigned)local);
    }
  }
}

// ------------------------------------------------------------ dispatch
struct BatchCfg {
  const char* name;
  int tx, ty, tz;
  const void* k64;
  const void* kmx;
};

#define BCFG(TX, TY, TZ, MINB)                                                       \
  { #TX "x" #TY "x" #TZ "/" #MINB, TX, TY, TZ,                                      \
    (const void*)batch_stage_fp64_kernel<TY, TZ, MINB>,                             \
    (const void*)batch_stage_kernel<TX, TY, TZ, MINB> }
static const BatchCfg k_bcfg[] = {
    BCFG(32, 8, 1, 1), BCFG(32, 2, 2, 2), BCFG(32, 4, 1, 3), BCFG(32, 4, 2, 1),
};
#undef BCFG

// one-block-per-tile configurations
struct TileCfgB {
  const char* name;
  int tx, ty, tz;
  const void* k64full;
  const void* k64;
  const void* kmx;
};
#define TCFG(TX, TY, TZ, MINB)                                                      \
  { "tiles" #TX "x" #TY "x" #TZ "/" #MINB, TX, TY, TZ,                            \
    (const void*)batch_tile_kernel<TX, TY, TZ, MINB, false, true>,                \
    (const void*)batch_tile_kernel<TX, TY, TZ, MINB, false, false>,               \
    (const void*)batch_tile_kernel<TX, TY, TZ, MINB, true, false> }
static const TileCfgB k_tcfg[] = {TCFG(32, 4, 1, 2), TCFG(32, 8, 1, 1)};
#undef TCFG

constexpr int N_FUSED = (int)(sizeof(k_bcfg) / sizeof(k_bcfg[0]));
constexpr int N_TILE = (int)(sizeof(k_tcfg) / sizeof(k_tcfg[0]));
constexpr int C_TMA = N_FUSED + N_TILE;  // then C_TMA + 1: the 11-field TMA variant
constexpr int N_TMA_B = 2;
// per-member launches of the single-grid kernels, the members' chains on 16,
// 4 or 1 auxiliary streams
constexpr int C_MEMB = C_TMA + N_TMA_B;
constexpr int N_MEMB = 3;
constexpr int k_memb_streams[N_MEMB] = {16, 4, 1};

int batch_tile_config_count() { return C_MEMB + N_MEMB + batch_ff_config_count(); }
int batch_ff_cfg_index(int v) { return C_MEMB + N_MEMB + v; }
int batch_ff_variant(int cfg) {
  const int v = cfg - (C_MEMB + N_MEMB);
  return (v >= 0 && v < batch_ff_config_count()) ? v : -1;
}
bool batch_tile_is_members(int c) { return c >= C_MEMB && c < C_MEMB + N_MEMB; }
int batch_members_streams(int c) { return batch_tile_is_members(c) ? k_memb_streams[c - C_MEMB] : 0; }
int batch_tma_variant(int cfg) {
  const int v = cfg - C_TMA;
  return (v >= 0 && v < N_TMA_B) ? v : -1;
}
// Default tile of a new batch (the serving loop keeps it): the fastest
// configuration of the 64-binary batched workload on GB300, for mixed and
// float64 batches alike the per-member launches of the single-grid kernels
// (whole steps over the 64 members: mixed 114.4 ms against 146.5 for the
// eleven-field persistent TMA kernel; float64 843.8 against 867.8 for
// tiles32x4x1/2 and 884.4 for the persistent 32x4x1/3).
int batch_default_tile(bool) { return C_MEMB; }
// double-word batches: the per-member chains one after another on a single
// stream (89.1 M point-updates/s over the 64 binaries against 73.9 for
// fftiles32x4x1/8+8 and 71.7 for chains on 16 streams, where different
// double-word kernels sharing an SM's instruction cache slow each other)
int batch_default_tile_ff() { return C_MEMB + 2; }
bool batch_tile_is_tma(int c) { return batch_tma_variant(c) >= 0; }
bool batch_tile_is_per_tile(int c) { return (c >= N_FUSED && c < C_TMA) || batch_ff_variant(c) >= 0; }
const char* batch_tile_config_name(int c) {
  if (batch_ff_variant(c) >= 0) return batch_ff_config_name(batch_ff_variant(c));
  if (c == C_TMA) return "tma32x4x1/2";
  if (c == C_TMA + 1) return "tma11_32x8x1/1";
  if (c == C_MEMB) return "members";
  if (c == C_MEMB + 1) return "members4";
  if (c == C_MEMB + 2) return "members1";
  if (batch_tile_is_per_tile(c)) return k_tcfg[c - N_FUSED].name;
  return (c >= 0 && c < N_FUSED) ? k_bcfg[c].name : "";
}
void batch_tile_shape(int c, int& tx, int& ty, int& tz) {
  if (batch_ff_variant(c) >= 0) {
    batch_ff_tile_shape(batch_ff_variant(c), tx, ty, tz);
    return;
  }
  if (batch_tma_variant(c) >= 0 || batch_tile_is_members(c)) {  // members: the 11-field TMA kernel's tiles
    batch_tma_tile_shape(batch_tile_is_members(c) ? 1 : batch_tma_variant(c), tx, ty, tz);
    return;
  }
  if (batch_tile_is_per_tile(c)) {
    const TileCfgB& t = k_tcfg[c - N_FUSED];
    tx = t.tx;
    ty = t.ty;
    tz = t.tz;
    return;
  }
  if (c < 0 || c >= N_FUSED) c = 0;
  tx = k_bcfg[c].tx;
  ty = k_bcfg[c].ty;
  tz = k_bcfg[c].tz;
}

bool batch_tile_full(int cfg, const Grid& g) {
  int tx, ty, tz;
  batch_tile_shape(cfg, tx, ty, tz);
  return tx == 32 && g.n0 % 32 == 0 && g.n1 % ty == 0 && g.n2 % tz == 0;
}

cudaError_t launch_batch_stage(int cfg, bool mixed, bool full, const MemberDev* mem, const BatchWork* wk,
                               unsigned ntiles, int stage, int* err, cudaStream_t s) {
  if (batch_tma_variant(cfg) >= 0 && mixed) return launch_batch_stage_tma(batch_tma_variant(cfg), mem, wk, stage, err, s);
  if (batch_tile_is_per_tile(cfg) && batch_ff_variant(cfg) < 0) {
    const TileCfgB& c = k_tcfg[cfg - N_FUSED];
    if (ntiles == 0) return cudaSuccess;
    full = full && !mixed;
    const void* fn = mixed ? c.kmx : (full ? c.k64full : c.k64);
    const size_t smem = full ? rows_block_smem(c.ty, c.tz, true) : 0;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    dim3 block(c.tx, c.ty, c.tz);
    void* args[] = {(void*)&mem, (void*)&wk, (void*)&stage};
    return cudaLaunchKernel(fn, dim3(ntiles), block, args, smem, s);
  }
  if (cfg < 0 || cfg >= N_FUSED) cfg = 0;
  const BatchCfg& c = k_bcfg[cfg];
  const void* fn = mixed ? c.kmx : c.k64;
  const int threads = c.tx * c.ty * c.tz;
  // float64 full-block tiles exchange first differences through shared memory
  const size_t smem = (!mixed && c.tx == 32) ? rows_block_smem(c.ty, c.tz, true) : 0;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = smem > 48 * 1024 ? cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                                   : cudaSuccess;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) per = 1;
  dim3 block(c.tx, c.ty, c.tz);
  dim3 grid((unsigned)(sms * per));
  void* args[] = {(void*)&mem, (void*)&wk, (void*)&stage};
  return cudaLaunchKernel(fn, grid, block, args, smem, s);
}

cudaError_t launch_batch_boundary(bool mixed, const MemberDev* mem, const BatchWork* wk, int stage,
                                  cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)(sms * 8)), block(256);
  // mixed Sommerfeld: four field groups per ghost point (gridDim.y); periodic
  // members copy every field in the first group and nothing in the others
  if (mixed) batch_boundary_kernel<true><<<dim3(grid.x, 4), block, 0, s>>>(mem, wk, stage);
  else batch_boundary_kernel<false><<<grid, block, 0, s>>>(mem, wk, stage);
  return cudaGetLastError();
}

}  // namespace bssn
