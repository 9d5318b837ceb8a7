// Device-side tables of a batch of evolutions (see bssn_batch.cu).
#pragma once
#include "bssn_internal.cuh"

namespace bssn {

constexpr int BATCH_MAX = BSSN_BATCH_MAX_MEMBERS;

// One member as the batched kernels see it: its grid and the arguments of its
// four RK4 stages (pointer roles fixed, y_n advanced in place).
struct MemberDev {
  Grid g;
  StageArgs a64[4];
  StageArgsMixed amx[4];
  int tiles[3];  // stage tiles per axis for the batch's current tile shape
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

int batch_tile_config_count();
const char* batch_tile_config_name(int c);
void batch_tile_shape(int c, int& tx, int& ty, int& tz);
// Persistent stage kernel over every active member's tiles (grid = blocks).
cudaError_t launch_batch_stage(int cfg, bool mixed, const MemberDev* mem, const BatchWork* wk,
                               int stage, cudaStream_t s);
// Boundary of every active member after a stage (Sommerfeld or periodic).
cudaError_t launch_batch_boundary(bool mixed, const MemberDev* mem, const BatchWork* wk, int stage,
                                  cudaStream_t s);

}  // namespace bssn
