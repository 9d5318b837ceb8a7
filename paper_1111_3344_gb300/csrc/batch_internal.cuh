// Device-side tables of a batch of evolutions (see bssn_batch.cu).
#pragma once
#include "bssn_internal.cuh"

namespace bssn {

constexpr int BATCH_MAX = BSSN_BATCH_MAX_MEMBERS;
// work lists of a batch: every active member (boundary, persistent and TMA
// stage kernels); float64 members with full tiles and the others (the
// one-block-per-tile stage kernels, one point function each)
constexpr int WORK_ALL = 0, WORK_FULL = 1, WORK_REST = 2, NWORK = 3;

// One member as the batched kernels see it: its grid and the arguments of its
// four RK4 stages (pointer roles fixed, y_n advanced in place).
struct MemberDev {
  Grid g;
  StageArgs a64[4];
  StageArgsMixed amx[4];
  StageArgsFF aff[4];  // double-word batches
  int tiles[3];  // stage tiles per axis for the batch's current tile shape
  // mixed: tensor map of each stage's input float buffer (TMA-staged batch
  // kernel); 64-byte aligned, as the tensor loads require
  CUtensorMap tmap[4];
};

// The active members and prefix sums of their work (rebuilt on the host when
// the composition changes; the captured graph reads it from device memory).
struct BatchWork {
  int count;
  unsigned total_tiles;
  unsigned long long total_bc;
  int member[BATCH_MAX];
  unsigned tile_base[BATCH_MAX + 1];
  unsigned long long bc_base[BATCH_MAX + 1];
};

// The boundary work list of a batch copied to shared memory by every block of
// a boundary kernel (prefix sums of the boundary items and the member of each
// slot, at most 3 KB), so that the member search of each item reads shared
// memory instead of a chain of dependent global loads.
struct BcList {
  unsigned long long base[BATCH_MAX + 1];
  int member[BATCH_MAX];
};
// every thread of the (one-dimensional) block calls this before its item loop
__device__ __forceinline__ void load_bc_list(BcList& L, const BatchWork* __restrict__ wk, int count) {
  for (int i = threadIdx.x; i <= count; i += blockDim.x) L.base[i] = wk->bc_base[i];
  for (int i = threadIdx.x; i < count; i += blockDim.x) L.member[i] = wk->member[i];
  __syncthreads();
}
// slot of boundary item t: the largest slot with base[slot] <= t
__device__ __forceinline__ int find_bc(const BcList& L, int count, unsigned long long t) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (L.base[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Tile configurations of the batched stage: persistent fused kernels (both
// precisions), one-block-per-tile fused kernels (both precisions), the two
// TMA-staged kernels (mixed only), then the double-word configurations.
int batch_tile_config_count();
const char* batch_tile_config_name(int c);
void batch_tile_shape(int c, int& tx, int& ty, int& tz);
bool batch_tile_is_tma(int c);
bool batch_tile_is_per_tile(int c);
int batch_default_tile(bool mixed);
// The per-member configurations ("members", "members4", "members1"): each member's stages run as
// launches of the single-grid stage and boundary kernels (the float64 32x4x1/1
// tiles, the mixed 11-field TMA kernel, the double-word ffrows32x4x1/8), the
// members' launch chains side by side on auxiliary streams (bssn_batch.cu).
bool batch_tile_is_members(int c);
// auxiliary streams the members' chains of configuration c are spread over
// ("members" 16, "members4" 4, "members1" 1; 0 for other configurations)
int batch_members_streams(int c);
int batch_default_tile_ff();
// Whether a float64 member has full tiles under configuration cfg (n0 a
// multiple of 32 = the tile's x extent, n1 and n2 of its y and z extents).
bool batch_tile_full(int cfg, const Grid& g);
// Stage kernel over the tiles of one work list.  Persistent and TMA-staged
// configurations: grid = resident blocks, every member (WORK_ALL).
// One-block-per-tile configurations: grid = ntiles, the list's tile count;
// full selects the full-block float64 point function (WORK_FULL).  err: device
// error word (a bounded wait of the TMA kernel gave up).
cudaError_t launch_batch_stage(int cfg, bool mixed, bool full, const MemberDev* mem, const BatchWork* wk,
                               unsigned ntiles, int stage, int* err, cudaStream_t s);
// TMA-staged forms (k_batch_tma.cu), variant v: 0 = 32x4x1 tiles with 8
// staged fields, 1 = 32x8x1 tiles with 11; batch_tma_variant(cfg): the
// variant of configuration cfg, -1 for the others
int batch_tma_variant(int cfg);
void batch_tma_tile_shape(int v, int& tx, int& ty, int& tz);
cudaError_t prepare_batch_stage_tma(int v);
cudaError_t launch_batch_stage_tma(int v, const MemberDev* mem, const BatchWork* wk, int stage, int* err,
                                   cudaStream_t s);
// Boundary of every active member after a stage (Sommerfeld or periodic).
cudaError_t launch_batch_boundary(bool mixed, const MemberDev* mem, const BatchWork* wk, int stage,
                                  cudaStream_t s);
// Double-word batches (k_batch_ff.cu): one-block-per-tile configurations v in
// [0, batch_ff_config_count()), their tile shapes, the stage launch over one
// work list (full: the members with full tiles) and the boundary launch.
int batch_ff_config_count();
const char* batch_ff_config_name(int v);
void batch_ff_tile_shape(int v, int& tx, int& ty, int& tz);
cudaError_t launch_batch_stage_ff(int v, bool full, const MemberDev* mem, const BatchWork* wk, unsigned ntiles,
                                  int stage, cudaStream_t s);
cudaError_t launch_batch_boundary_ff(const MemberDev* mem, const BatchWork* wk, int stage, cudaStream_t s);
// index of double-word configuration v in the batch's configuration list, and
// the inverse (-1 for other configurations)
int batch_ff_cfg_index(int v);
int batch_ff_variant(int cfg);

}  // namespace bssn
