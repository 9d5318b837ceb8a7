// Batches of independent evolutions advanced together (one persistent launch
// per RK4 stage under a captured CUDA graph) and the continuous-batching
// server built on them.
//
// A batch owns nothing but host bookkeeping: every device byte comes from the
// pool the caller passes (tables, then member registers carved by a first-fit
// sub-allocator).  The graph of one RK4 step is captured once per tile shape;
// it reads the member table and the work-list from device memory, so members
// can join and leave between steps without re-capture.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "batch_internal.cuh"

using namespace bssn;

namespace {

constexpr size_t ALIGN = 256;
size_t aup(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

bssn_status bfail(bssn_status s, const std::string& m) {
  set_last_error(m);
  return s;
}
bssn_status bcuda(cudaError_t e, const char* where) {
  return bfail(BSSN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// First-fit sub-allocator over [0, size) with coalescing frees.
struct Pool {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t base, size_t sz) {
    size = sz;
    free_.clear();
    if (sz > base) free_[base] = sz - base;
  }
  bool alloc(size_t n, size_t& off) {
    n = aup(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        off = it->first;
        const size_t rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = aup(n);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// Register layout of one member inside its pool block.
struct MemberLayout {
  size_t yn, ks, s1, s2, ksh;      // float64 path (ks, ksh also double-word)
  size_t gtab;                     // float64 Sommerfeld: ghost-geometry table (per-member chains)
  bool has_gtab;
  size_t m32[3], mw[3], ks32, ksw; // mixed path
  size_t f2[3];                    // double-word path: stage buffers (f2[0] the shadow of y_n)
  size_t part, out16, total;
  int nblocks;
};

MemberLayout member_layout(const bssn_params* p, const Grid& g) {
  MemberLayout L{};
  const size_t regb = aup((size_t)NF * g.fstride * sizeof(double));
  const size_t reg32 = aup((size_t)NF * g.fstride * sizeof(float));
  const size_t wb = aup((size_t)g.fstride * sizeof(double));
  const bool som = p->boundary == BSSN_BC_SOMMERFELD;
  size_t o = 0;
  L.yn = o; o += regb;
  if (p->precision == BSSN_FP64) {
    L.ks = o; o += regb;
    L.s1 = o; o += regb;
    L.s2 = o; o += regb;
    L.ksh = o; if (som) o += regb;
    L.has_gtab = som;
    L.gtab = o; if (som) o += aup(ghost_table_size(g));
  } else if (p->precision == BSSN_FF) {
    L.ks = o; o += regb;
    for (int q = 0; q < 3; q++) {
      L.f2[q] = o; o += regb;
    }
    L.ksh = o; if (som) o += regb;
  } else {
    for (int q = 0; q < 3; q++) {
      L.m32[q] = o; o += reg32;
      L.mw[q] = o; o += wb;
    }
    L.ks32 = o; o += reg32;
    L.ksw = o; o += wb;
    L.ksh = o; if (som) o += reg32;
  }
  L.nblocks = constraints_blocks(g);
  L.part = o; o += aup((size_t)L.nblocks * 18 * sizeof(double));
  L.out16 = o; o += aup(16 * sizeof(double));
  L.total = o;
  return L;
}

struct Member {
  bool used = false, active = false;
  bool held = false;  // resident but left out of the steps (bssn_batch_hold)
  bssn_params p{};
  Grid g{};
  MemberLayout L{};
  size_t off = 0;
  double t = 0.0;
  int npunct = 0;
  double punct[8][4] = {};
  long long steps = 0;
};

}  // namespace

struct bssn_batch {
  int precision;
  int maxm;
  cudaStream_t stream;
  char* pool;
  size_t pool_bytes;
  Pool alloc;
  std::vector<Member> m;
  MemberDev* d_mem;
  BatchWork* d_work;  // NWORK lists (batch_internal.cuh)
  int* d_err;          // error word of the TMA-staged kernel's bounded waits
  bool tma_ok = true;  // every member's tensor maps could be encoded
  int stall_polls = 0;  // test hook of the TMA-staged kernel (bssn_batch_test_stall_tma)
  std::vector<MemberDev> h_mem;
  BatchWork h_work[NWORK];
  bool work_dirty = true;
  int cfg = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // per-member configuration: auxiliary streams the members' launch chains
  // are spread over, and the events that fork them from and join them to
  // the batch's stream (made when the configuration is first selected)
  static constexpr int NAUX = 16;
  cudaStream_t aux[NAUX] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[NAUX] = {};
  bool aux_ok = false;
  std::mutex mu;  // guards everything above against concurrent API calls
};

namespace {

char* mptr(bssn_batch* b, const Member& M, size_t off) { return b->pool + M.off + off; }

void fill_member_dev(bssn_batch* b, int id) {
  Member& M = b->m[id];
  MemberDev& D = b->h_mem[id];
  memset(&D, 0, sizeof(D));
  D.g = M.g;
  int tx, ty, tz;
  batch_tile_shape(b->cfg, tx, ty, tz);
  D.tiles[0] = (M.g.n0 + tx - 1) / tx;
  D.tiles[1] = (M.g.n1 + ty - 1) / ty;
  D.tiles[2] = (M.g.n2 + tz - 1) / tz;
  const double dt = M.p.dt;
  const double a_dt[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
  const double b_dt[4] = {0.0, 0.0, 0.0, dt / 6.0};
  const int mode[4] = {MODE_FIRST, MODE_MID, MODE_MID, MODE_LAST};
  const bool som = M.p.boundary == BSSN_BC_SOMMERFELD;
  if (b->precision == BSSN_FP64) {
    double* yn = (double*)mptr(b, M, M.L.yn);
    double* s1 = (double*)mptr(b, M, M.L.s1);
    double* s2 = (double*)mptr(b, M, M.L.s2);
    double* src[4] = {yn, s1, s2, s1};
    double* out[4] = {s1, s2, s1, nullptr};
    for (int s = 0; s < 4; s++) {
      StageArgs& a = D.a64[s];
      a.src = src[s];
      a.src0 = yn;
      a.yn = yn;
      a.out0 = out[s];
      a.ksum = (double*)mptr(b, M, M.L.ks);
      a.kshell = som ? (double*)mptr(b, M, M.L.ksh) : nullptr;
      a.a_dt = a_dt[s];
      a.b_dt = b_dt[s];
      a.mode = mode[s];
    }
  } else if (b->precision == BSSN_FF) {
    const int src[4] = {0, 1, 2, 1}, out[4] = {1, 2, 1, 0};
    for (int s = 0; s < 4; s++) {
      StageArgsFF& a = D.aff[s];
      a.src = (const float2*)mptr(b, M, M.L.f2[src[s]]);
      a.src0 = (const float2*)mptr(b, M, M.L.f2[0]);
      a.yn = (double*)mptr(b, M, M.L.yn);
      a.out0 = (float2*)mptr(b, M, M.L.f2[out[s]]);
      a.ksum = (double*)mptr(b, M, M.L.ks);
      a.kshell = som ? (float2*)mptr(b, M, M.L.ksh) : nullptr;
      a.a_dt = a_dt[s];
      a.b_dt = b_dt[s];
      a.a_hi = (float)a_dt[s];
      a.a_lo = (float)(a_dt[s] - (double)a.a_hi);
      a.mode = mode[s];
    }
  } else {
    const int src[4] = {0, 1, 2, 1}, out[4] = {1, 2, 1, 0};
    for (int s = 0; s < 4; s++) {
      StageArgsMixed& a = D.amx[s];
      a.src = (float*)mptr(b, M, M.L.m32[src[s]]);
      a.srcw = (double*)mptr(b, M, M.L.mw[src[s]]);
      a.src0 = (float*)mptr(b, M, M.L.m32[0]);
      a.src0w = (double*)mptr(b, M, M.L.mw[0]);
      a.yn = (double*)mptr(b, M, M.L.yn);
      a.out0 = (float*)mptr(b, M, M.L.m32[out[s]]);
      a.out0w = (double*)mptr(b, M, M.L.mw[out[s]]);
      a.ksum = (float*)mptr(b, M, M.L.ks32);
      a.ksumw = (double*)mptr(b, M, M.L.ksw);
      a.kshell = som ? (float*)mptr(b, M, M.L.ksh) : nullptr;
      a.a_dt = a_dt[s];
      a.a_dtf = (float)a_dt[s];
      a.b_dt = b_dt[s];
      a.w_thr = M.p.w_fp64_threshold;
      a.mode = mode[s];
      a.stall_polls = b->stall_polls;
      // the box of the batch's TMA variant (32x8x1 tiles: tensor-map variant 1)
      const bool box8 = batch_tma_variant(b->cfg) == 1 || batch_tile_is_members(b->cfg);
      if (make_stage_tensor_map(M.g, a.src, &D.tmap[s], box8 ? 1 : 0) != cudaSuccess)
        b->tma_ok = false;
    }
  }
}

cudaError_t upload_member(bssn_batch* b, int id) {
  return cudaMemcpyAsync(b->d_mem + id, &b->h_mem[id], sizeof(MemberDev), cudaMemcpyHostToDevice,
                         b->stream);
}

cudaError_t rebuild_work(bssn_batch* b) {
  for (int w = 0; w < NWORK; w++) {
    BatchWork& W = b->h_work[w];
    W.count = 0;
    W.total_tiles = 0;
    W.total_bc = 0;
  }
  unsigned tb[NWORK] = {0, 0, 0};
  unsigned long long bb = 0;
  for (int id = 0; id < b->maxm; id++) {
    const Member& M = b->m[id];
    if (!M.used || !M.active || M.held) continue;
    const MemberDev& D = b->h_mem[id];
    const unsigned tiles = (unsigned)D.tiles[0] * D.tiles[1] * D.tiles[2];
    const int v = batch_tile_full(b->cfg, M.g) ? WORK_FULL : WORK_REST;
    for (int w : {WORK_ALL, v}) {
      BatchWork& W = b->h_work[w];
      W.member[W.count] = id;
      W.tile_base[W.count] = tb[w];
      if (w == WORK_ALL) W.bc_base[W.count] = bb;
      tb[w] += tiles;
      W.count++;
    }
    bb += ghost_count(M.g);  // one thread per ghost point (every field)
  }
  for (int w = 0; w < NWORK; w++) {
    BatchWork& W = b->h_work[w];
    W.tile_base[W.count] = tb[w];
    W.total_tiles = tb[w];
  }
  BatchWork& A = b->h_work[WORK_ALL];
  A.bc_base[A.count] = bb;
  A.total_bc = bb;
  b->work_dirty = false;
  // the one-block-per-tile kernels are captured with the lists' tile counts as
  // their grids: the graph is made again for the new composition
  if (batch_tile_is_per_tile(b->cfg) || batch_tile_is_members(b->cfg)) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->graph) {
      cudaGraphDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  return cudaMemcpyAsync(b->d_work, b->h_work, sizeof(b->h_work), cudaMemcpyHostToDevice, b->stream);
}

// ---- per-member configuration
// the single-grid configurations it launches (looked up by name once)
int single_fp64_cfg() {
  static int c = -1;
  if (c < 0)
    for (int q = 0; q < tile_config_count(); q++)
      if (!strcmp(tile_config_name(q), "32x4x1/1")) c = q;
  return c < 0 ? 0 : c;
}
int single_ff_cfg() {
  static int c = -1;
  if (c < 0)
    for (int q = 0; q < ff_config_count(); q++)
      if (!strcmp(ff_config_name(q), "ffrows32x4x1/8")) c = q;
  return c < 0 ? 0 : c;
}

void destroy_aux(bssn_batch* b) {
  for (int k = 0; k < bssn_batch::NAUX; k++) {
    if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    b->aux[k] = nullptr;
    b->ev_join[k] = nullptr;
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  b->ev_fork = nullptr;
  b->aux_ok = false;
}

// the auxiliary streams and events, made once; a partial failure releases
// what was made, so that a later call starts again from nothing
cudaError_t ensure_aux(bssn_batch* b) {
  if (b->aux_ok) return cudaSuccess;
  cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int k = 0; k < bssn_batch::NAUX && e == cudaSuccess; k++) {
    e = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    destroy_aux(b);
    return e;
  }
  b->aux_ok = true;
  return cudaSuccess;
}

// member id's stage with the single-grid stage kernel of the batch's precision
cudaError_t member_stage(bssn_batch* b, int id, int stage, cudaStream_t s) {
  const MemberDev& D = b->h_mem[id];
  if (b->precision == BSSN_MIXED) return launch_stage_mixed_tma(D.g, D.amx[stage], D.tmap[stage], b->d_err, s, 2);
  if (b->precision == BSSN_FF) return launch_stage_ff(D.g, D.aff[stage], s, single_ff_cfg());
  return launch_stage_fp64(D.g, D.a64[stage], s, single_fp64_cfg());
}

// member id's boundary after a stage, with the single-grid boundary kernels
// (the same per-point operations as the batched boundary kernel)
cudaError_t member_boundary(bssn_batch* b, int id, int stage, cudaStream_t s) {
  const MemberDev& D = b->h_mem[id];
  const Grid& g = D.g;
  if (b->precision == BSSN_MIXED) {
    const StageArgsMixed& a = D.amx[stage];
    if (!g.periodic) return launch_sommerfeld_mixed(g, a, a.kshell, s);
    cudaError_t e = launch_periodic_fill_mixed(g, a.out0, a.out0w, s);
    return (e == cudaSuccess && a.mode == MODE_LAST) ? launch_periodic_fill(g, a.yn, s) : e;
  }
  if (b->precision == BSSN_FF) {
    const StageArgsFF& a = D.aff[stage];
    if (!g.periodic) return launch_sommerfeld_ff(g, a, a.kshell, s);
    // the copy moves 8-byte values whatever they hold
    cudaError_t e = launch_periodic_fill(g, reinterpret_cast<double*>(a.out0), s);
    return (e == cudaSuccess && a.mode == MODE_LAST) ? launch_periodic_fill(g, a.yn, s) : e;
  }
  const StageArgs& a = D.a64[stage];
  const Member& M = b->m[id];
  if (!g.periodic) return launch_sommerfeld(g, a, a.kshell, s, M.L.has_gtab ? mptr(b, M, M.L.gtab) : nullptr);
  return launch_periodic_fill(g, a.mode == MODE_LAST ? a.yn : a.out0, s);
}

// Stages [s0, s1) of every active member: each member's chain (stage, then its
// boundary when bc) on auxiliary stream (slot % NAUX), forked from and joined
// back to the batch's stream, so that different members' kernels overlap.
cudaError_t launch_members(bssn_batch* b, int s0, int s1, bool bc) {
  cudaError_t e = cudaEventRecord(b->ev_fork, b->stream);
  for (int k = 0; k < bssn_batch::NAUX && e == cudaSuccess; k++) e = cudaStreamWaitEvent(b->aux[k], b->ev_fork, 0);
  const BatchWork& W = b->h_work[WORK_ALL];
  const int nstreams = batch_members_streams(b->cfg);
  for (int slot = 0; slot < W.count && e == cudaSuccess; slot++) {
    cudaStream_t s = b->aux[slot % nstreams];
    for (int st = s0; st < s1 && e == cudaSuccess; st++) {
      e = member_stage(b, W.member[slot], st, s);
      if (e == cudaSuccess && bc) e = member_boundary(b, W.member[slot], st, s);
    }
  }
  // join every auxiliary stream back, even after a failed launch, so that the
  // batch's stream orders whatever was issued on them
  for (int k = 0; k < bssn_batch::NAUX; k++) {
    cudaError_t j = cudaEventRecord(b->ev_join[k], b->aux[k]);
    if (j == cudaSuccess) j = cudaStreamWaitEvent(b->stream, b->ev_join[k], 0);
    if (e == cudaSuccess) e = j;
  }
  return e;
}

// The stage launches of one RK4 stage under configuration cfg: persistent and
// TMA-staged kernels, one launch over every member; one-block-per-tile
// kernels, one launch per float64 list (members with full tiles, the others),
// or one over every member (mixed).
cudaError_t launch_stage_lists(bssn_batch* b, int cfg, int stage) {
  if (batch_tile_is_members(cfg)) return launch_members(b, stage, stage + 1, false);
  const bool mixed = b->precision == BSSN_MIXED;
  if (b->precision == BSSN_FF) {
    const int v = batch_ff_variant(cfg);
    cudaError_t e = launch_batch_stage_ff(v, true, b->d_mem, b->d_work + WORK_FULL, b->h_work[WORK_FULL].total_tiles,
                                          stage, b->stream);
    if (e == cudaSuccess)
      e = launch_batch_stage_ff(v, false, b->d_mem, b->d_work + WORK_REST, b->h_work[WORK_REST].total_tiles, stage,
                                b->stream);
    return e;
  }
  if (!batch_tile_is_per_tile(cfg) || mixed)
    return launch_batch_stage(cfg, mixed, false, b->d_mem, b->d_work + WORK_ALL, b->h_work[WORK_ALL].total_tiles,
                              stage, b->d_err, b->stream);
  cudaError_t e = launch_batch_stage(cfg, false, true, b->d_mem, b->d_work + WORK_FULL,
                                     b->h_work[WORK_FULL].total_tiles, stage, b->d_err, b->stream);
  if (e == cudaSuccess)
    e = launch_batch_stage(cfg, false, false, b->d_mem, b->d_work + WORK_REST, b->h_work[WORK_REST].total_tiles,
                           stage, b->d_err, b->stream);
  return e;
}

cudaError_t capture(bssn_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const bool mixed = b->precision == BSSN_MIXED;
  // per-member configuration: each member's whole step (4 stages and their
  // boundaries) as one chain, the chains side by side
  if (batch_tile_is_members(b->cfg)) e = launch_members(b, 0, 4, true);
  for (int s = 0; s < 4 && e == cudaSuccess && !batch_tile_is_members(b->cfg); s++) {
    e = launch_stage_lists(b, b->cfg, s);
    if (e == cudaSuccess)
      e = b->precision == BSSN_FF ? launch_batch_boundary_ff(b->d_mem, b->d_work + WORK_ALL, s, b->stream)
                                  : launch_batch_boundary(mixed, b->d_mem, b->d_work + WORK_ALL, s, b->stream);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  b->graph = g;
  return cudaGraphInstantiate(&b->exec, g, 0);
}

// prepare a member's registers after its y_n was written (periodic ghosts,
// float shadow for the mixed path)
cudaError_t after_state(bssn_batch* b, Member& M) {
  double* yn = (double*)mptr(b, M, M.L.yn);
  cudaError_t e = cudaSuccess;
  if (M.g.periodic) e = launch_periodic_fill(M.g, yn, b->stream);
  if (e == cudaSuccess && b->precision == BSSN_MIXED)
    e = launch_shadow(M.g, yn, (float*)mptr(b, M, M.L.m32[0]), (double*)mptr(b, M, M.L.mw[0]), b->stream);
  if (e == cudaSuccess && b->precision == BSSN_FF)
    e = launch_shadow_ff(M.g, yn, (float2*)mptr(b, M, M.L.f2[0]), b->stream);
  return e;
}

bool member_ok(bssn_batch* b, int id) { return b && id >= 0 && id < b->maxm && b->m[id].used; }

bool tile_usable(const bssn_batch* b, int c) {
  if (batch_tile_is_members(c)) return b->precision != BSSN_MIXED || b->tma_ok;
  if ((batch_ff_variant(c) >= 0) != (b->precision == BSSN_FF)) return false;
  return !batch_tile_is_tma(c) || (b->precision == BSSN_MIXED && b->tma_ok);
}

// Switch the batch to tile configuration cfg (stream idle): member tables
// refilled and uploaded, work list and graph rebuilt at the next step.
// What configuration cfg needs before its first launch (outside graph capture):
// the TMA kernels' shared-memory limit, the per-member configuration's streams.
cudaError_t prepare_cfg(bssn_batch* b, int cfg) {
  cudaError_t e = batch_tile_is_tma(cfg) ? prepare_batch_stage_tma(batch_tma_variant(cfg)) : cudaSuccess;
  if (e == cudaSuccess && batch_tile_is_members(cfg)) {
    e = ensure_aux(b);
    if (e == cudaSuccess && b->precision == BSSN_MIXED) e = prepare_stage_mixed_tma(2);
  }
  return e;
}

cudaError_t apply_cfg(bssn_batch* b, int cfg) {
  cudaError_t e = prepare_cfg(b, cfg);
  if (e != cudaSuccess) return e;
  b->cfg = cfg;
  for (int id = 0; id < b->maxm && e == cudaSuccess; id++)
    if (b->m[id].used) {
      fill_member_dev(b, id);
      e = upload_member(b, id);
    }
  b->work_dirty = true;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  return e;
}

// After a synchronisation: did a stage kernel give up waiting for its tile?
// (the states it touched are invalid); the word is cleared.
bssn_status check_batch_err(bssn_batch* b) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch error word");
  if (h) {
    cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
    return bfail(BSSN_ETIMEOUT, "a batched stage kernel gave up waiting for its shared-memory tile; the states are invalid");
  }
  return BSSN_OK;
}

}  // namespace

extern "C" {

size_t bssn_batch_member_bytes(const bssn_params* p) {
  std::string why;
  if (!validate_params(p, why)) {
    set_last_error(why);
    return 0;
  }
  Grid g = grid_of(p);
  return member_layout(p, g).total;
}

size_t bssn_batch_table_bytes(int32_t max_members) {
  if (max_members < 1 || max_members > BATCH_MAX) return 0;
  return aup(sizeof(MemberDev) * (size_t)max_members) + aup(NWORK * sizeof(BatchWork)) + aup(sizeof(int));
}

bssn_status bssn_batch_create(int32_t precision, int32_t max_members, void* d_pool, size_t pool_bytes,
                              void* cuda_stream, bssn_batch** out) {
  if (!out) return bfail(BSSN_EINVAL, "out is NULL");
  *out = nullptr;
  if (precision != BSSN_FP64 && precision != BSSN_MIXED && precision != BSSN_FF)
    return bfail(BSSN_EINVAL, "bad precision");
  if (max_members < 1 || max_members > BATCH_MAX)
    return bfail(BSSN_EINVAL, "max_members must be 1.." + std::to_string(BATCH_MAX));
  if (!d_pool || ((uintptr_t)d_pool) % ALIGN) return bfail(BSSN_EINVAL, "d_pool must be non-NULL, 256-byte aligned");
  if (!cuda_stream) return bfail(BSSN_EINVAL, "a batch needs a non-default stream (graph capture)");
  const size_t tb = bssn_batch_table_bytes(max_members);
  if (pool_bytes < tb) return bfail(BSSN_ENOMEM, "pool smaller than the batch tables");
  bssn_batch* b = new (std::nothrow) bssn_batch();
  if (!b) return bfail(BSSN_ENOMEM, "host allocation failed");
  b->precision = precision;
  b->maxm = max_members;
  b->stream = (cudaStream_t)cuda_stream;
  b->pool = (char*)d_pool;
  b->pool_bytes = pool_bytes;
  b->alloc.init(tb, pool_bytes);
  b->m.resize(max_members);
  b->h_mem.resize(max_members);
  memset(b->h_work, 0, sizeof(b->h_work));
  b->d_mem = (MemberDev*)b->pool;
  b->d_work = (BatchWork*)(b->pool + aup(sizeof(MemberDev) * (size_t)max_members));
  b->d_err = (int*)((char*)b->d_work + aup(NWORK * sizeof(BatchWork)));
  b->cfg = precision == BSSN_FF ? batch_default_tile_ff() : batch_default_tile(precision == BSSN_MIXED);
  cudaError_t e = prepare_cfg(b, b->cfg);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = rebuild_work(b);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    destroy_aux(b);
    delete b;
    return bcuda(e, "batch create");
  }
  *out = b;
  return BSSN_OK;
}

bssn_status bssn_batch_free(bssn_batch* b) {
  if (!b) return bfail(BSSN_EINVAL, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  destroy_aux(b);
  delete b;
  if (e != cudaSuccess) return bcuda(e, "batch free");
  return BSSN_OK;
}

bssn_status bssn_batch_add(bssn_batch* b, const bssn_params* p, int32_t* member) {
  if (!b || !p || !member) return bfail(BSSN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(b->mu);
  std::string why;
  if (!validate_params(p, why)) return bfail(BSSN_EINVAL, why);
  if (p->precision != b->precision) return bfail(BSSN_EINVAL, "member precision differs from the batch's");
  if (p->ksum_fp64) return bfail(BSSN_EINVAL, "ksum_fp64 is for single-grid contexts");
  int id = -1;
  for (int q = 0; q < b->maxm; q++)
    if (!b->m[q].used) { id = q; break; }
  if (id < 0) return bfail(BSSN_ENOMEM, "batch is full");
  Member M;
  M.used = true;
  M.p = *p;
  M.g = grid_of(p);
  M.L = member_layout(p, M.g);
  if (!b->alloc.alloc(M.L.total, M.off))
    return bfail(BSSN_ENOMEM, "pool exhausted: member needs " + std::to_string(M.L.total) + " bytes");
  b->m[id] = M;
  fill_member_dev(b, id);
  cudaError_t e = upload_member(b, id);
  // float64 Sommerfeld members: the ghost-geometry table of the single-grid
  // boundary kernels (the per-member chains use them)
  if (e == cudaSuccess && M.L.has_gtab) e = launch_ghost_table(M.g, mptr(b, M, M.L.gtab), b->stream);
  // a member whose tensor maps could not be encoded: fall back to a fused tile
  // (the TMA-staged configurations, and the per-member one on the mixed path,
  // whose stage kernel is the TMA-staged one)
  const bool needs_maps =
      batch_tile_is_tma(b->cfg) || (batch_tile_is_members(b->cfg) && b->precision == BSSN_MIXED);
  if (e == cudaSuccess && !b->tma_ok && needs_maps) {
    e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = apply_cfg(b, 0);
  }
  if (e != cudaSuccess) return bcuda(e, "batch add");
  *member = id;
  return BSSN_OK;
}

bssn_status bssn_batch_remove(bssn_batch* b, int32_t id) {
  if (!b) return bfail(BSSN_EINVAL, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  if (!member_ok(b, id)) return bfail(BSSN_ENOTFOUND, "no such member");
  // in-flight graph replays may still read the member's registers
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch remove");
  Member& M = b->m[id];
  const bool was_active = M.active;
  b->alloc.release(M.off, M.L.total);
  M = Member();
  if (was_active) b->work_dirty = true;
  return BSSN_OK;
}

bssn_status bssn_batch_set_initial_data(bssn_batch* b, int32_t id, int32_t kind, const double* p,
                                        int32_t np) {
  if (!b) return bfail(BSSN_EINVAL, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  if (!member_ok(b, id)) return bfail(BSSN_ENOTFOUND, "no such member");
  if (np < 0 || (np > 0 && !p) || np > 33) return bfail(BSSN_EINVAL, "bad parameter array");
  Member& M = b->m[id];
  int npunct = 0;
  if (kind == BSSN_ID_BL) {
    if (np < 1) return bfail(BSSN_EINVAL, "BL needs {npunct, m, x, y, z, ...}");
    npunct = (int)p[0];
    if (npunct < 1 || npunct > 8 || (double)npunct != p[0] || np < 1 + 4 * npunct)
      return bfail(BSSN_EINVAL, "BL: npunct must be 1..8 with 4 values each");
  } else if (kind == BSSN_ID_GAUGE_WAVE) {
    if (np < 2 || !(p[1] != 0.0) || !(std::fabs(p[0]) < 1.0)) return bfail(BSSN_EINVAL, "gauge wave: {A, d}");
  } else if (kind == BSSN_ID_KASNER) {
    if (np < 1 || !(p[0] > 0.0)) return bfail(BSSN_EINVAL, "Kasner needs {t0 > 0}");
  } else if (kind != BSSN_ID_FLAT) {
    return bfail(BSSN_EINVAL, "unknown initial-data kind");
  }
  double* yn = (double*)mptr(b, M, M.L.yn);
  cudaError_t e = launch_initial_data(M.g, kind, p, np, yn, b->stream);
  if (e == cudaSuccess) e = after_state(b, M);
  if (e != cudaSuccess) return bcuda(e, "batch initial data");
  M.npunct = npunct;
  for (int a = 0; a < npunct; a++)
    for (int q = 0; q < 4; q++) M.punct[a][q] = p[1 + 4 * a + q];
  M.t = 0.0;
  M.steps = 0;
  if (!M.active) b->work_dirty = true;
  M.active = true;
  return BSSN_OK;
}

bssn_status bssn_batch_set_state(bssn_batch* b, int32_t id, const double* host, double t) {
  if (!b || !host) return bfail(BSSN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(b->mu);
  if (!member_ok(b, id)) return bfail(BSSN_ENOTFOUND, "no such member");
  Member& M = b->m[id];
  const Grid& g = M.g;
  double* yn = (double*)mptr(b, M, M.L.yn);
  cudaError_t e = cudaMemcpy2DAsync(yn, (size_t)g.pitch * 8, host, (size_t)g.sx * 8, (size_t)g.sx * 8,
                                    (size_t)NF * g.sz * g.sy, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = after_state(b, M);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch set_state");
  M.t = t;
  if (!M.active) b->work_dirty = true;
  M.active = true;
  return BSSN_OK;
}

bssn_status bssn_batch_get_state(bssn_batch* b, int32_t id, double* host, double* t) {
  if (!b || !host) return bfail(BSSN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(b->mu);
  if (!member_ok(b, id)) return bfail(BSSN_ENOTFOUND, "no such member");
  Member& M = b->m[id];
  const Grid& g = M.g;
  const double* yn = (const double*)mptr(b, M, M.L.yn);
  cudaError_t e = cudaMemcpy2DAsync(host, (size_t)g.sx * 8, yn, (size_t)g.pitch * 8, (size_t)g.sx * 8,
                                    (size_t)NF * g.sz * g.sy, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch get_state");
  if (bssn_status es = check_batch_err(b)) return es;
  if (t) *t = M.t;
  return BSSN_OK;
}

bssn_status bssn_batch_step(bssn_batch* b, int32_t nsteps) {
  if (!b) return bfail(BSSN_EINVAL, "batch is NULL");
  if (nsteps < 0) return bfail(BSSN_EINVAL, "nsteps < 0");
  std::lock_guard<std::mutex> lk(b->mu);
  cudaError_t e = cudaSuccess;
  if (b->work_dirty) e = rebuild_work(b);
  if (e == cudaSuccess && !b->exec) e = capture(b);
  if (e != cudaSuccess) return bcuda(e, "batch step setup");
  if (b->h_work[WORK_ALL].count == 0) return BSSN_OK;
  for (int s = 0; s < nsteps; s++) {
    e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return bcuda(e, "batch graph launch");
  }
  for (int id = 0; id < b->maxm; id++) {
    Member& M = b->m[id];
    if (M.used && M.active && !M.held) {
      M.t += nsteps * M.p.dt;
      M.steps += nsteps;
    }
  }
  return BSSN_OK;
}

bssn_status bssn_batch_hold(bssn_batch* b, int32_t id, int32_t hold) {
  if (!b) return bfail(BSSN_EINVAL, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  if (!member_ok(b, id)) return bfail(BSSN_ENOTFOUND, "no such member");
  Member& M = b->m[id];
  const bool h = hold != 0;
  if (M.held != h && M.active) b->work_dirty = true;
  M.held = h;
  return BSSN_OK;
}

int32_t bssn_serve_select(int32_t n, const double* remaining_work, const double* points, double min_points,
                          int32_t* selected) {
  if (n <= 0 || !remaining_work || !points || !selected) return 0;
  std::vector<int> order(n);
  for (int i = 0; i < n; i++) order[i] = i;
  // shortest remaining work first; ties by index, so the choice is deterministic
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return remaining_work[a] < remaining_work[c]; });
  for (int i = 0; i < n; i++) selected[i] = 0;
  double acc = 0.0;
  int32_t count = 0;
  for (int i = 0; i < n; i++) {
    if (count > 0 && acc >= min_points) break;
    selected[order[i]] = 1;
    acc += points[order[i]];
    count++;
  }
  return count;
}

bssn_status bssn_batch_constraints(bssn_batch* b, int32_t id, double out[16]) {
  if (!b || !out) return bfail(BSSN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(b->mu);
  if (!member_ok(b, id)) return bfail(BSSN_ENOTFOUND, "no such member");
  Member& M = b->m[id];
  double* dout = (double*)mptr(b, M, M.L.out16);
  cudaError_t e = launch_constraints(M.g, (const double*)mptr(b, M, M.L.yn), &M.punct[0][0], M.npunct,
                                     M.p.r_excise, (double*)mptr(b, M, M.L.part), M.L.nblocks, dout,
                                     b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, 16 * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch constraints");
  return check_batch_err(b);
}

bssn_status bssn_batch_test_stall_tma(bssn_batch* b, int32_t polls) {
  if (!b) return bfail(BSSN_EINVAL, "batch is NULL");
  if (polls < 0 || polls > (1 << 20)) return bfail(BSSN_EINVAL, "polls must be in [0, 2^20]");
  std::lock_guard<std::mutex> lk(b->mu);
  b->stall_polls = polls;
  // the captured graph reads the member tables from device memory: refill
  // and upload them in stream order, no re-capture (the per-member
  // configuration holds the arguments in its launches: captured again)
  cudaError_t e = cudaSuccess;
  for (int id = 0; id < b->maxm && e == cudaSuccess; id++)
    if (b->m[id].used) {
      fill_member_dev(b, id);
      e = upload_member(b, id);
    }
  if (e != cudaSuccess) return bcuda(e, "batch member tables");
  if (batch_tile_is_members(b->cfg)) b->work_dirty = true;
  return BSSN_OK;
}

int32_t bssn_batch_tile_count(void) { return batch_tile_config_count(); }
const char* bssn_batch_tile_name(int32_t c) { return batch_tile_config_name(c); }

bssn_status bssn_batch_set_tile(bssn_batch* b, int32_t cfg) {
  if (!b) return bfail(BSSN_EINVAL, "batch is NULL");
  std::lock_guard<std::mutex> lk(b->mu);
  if (cfg < 0 || cfg >= batch_tile_config_count()) return bfail(BSSN_EINVAL, "tile config out of range");
  if (!tile_usable(b, cfg))
    return bfail(BSSN_EINVAL, "tile not for this batch's precision (the TMA-staged tile is for mixed batches, "
                              "the fftiles ones for double-word batches)");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = apply_cfg(b, cfg);
  if (e != cudaSuccess) return bcuda(e, "set tile");
  return BSSN_OK;
}

bssn_status bssn_batch_autotune(bssn_batch* b, int32_t reps, int32_t* best, double* ms_per_cfg) {
  if (!b || reps < 1) return bfail(BSSN_EINVAL, "bad argument");
  const int n = batch_tile_config_count();
  double best_ms = 1e300;
  int best_c = 0;
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return bcuda(e, "event");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bcuda(e, "event");
  }
  bssn_status st = BSSN_OK;
  for (int c = 0; c < n && st == BSSN_OK; c++) {
    if (!tile_usable(b, c)) {
      if (ms_per_cfg) ms_per_cfg[c] = -1.0;
      continue;
    }
    if ((st = bssn_batch_set_tile(b, c)) != BSSN_OK) break;
    std::lock_guard<std::mutex> lk(b->mu);
    if (b->work_dirty && (e = rebuild_work(b)) != cudaSuccess) { st = bcuda(e, "autotune"); break; }
    // stages 0 and 1 write only stage buffers and the k-sum (y_n is left
    // unchanged, the next step overwrites them); the second stage carries the
    // combine's extra loads, which the first alone would not weigh
    auto pair = [&]() -> cudaError_t {
      cudaError_t r = launch_stage_lists(b, c, 0);
      return r == cudaSuccess ? launch_stage_lists(b, c, 1) : r;
    };
    e = pair();
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < reps && e == cudaSuccess; r++) e = pair();
    cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { st = bcuda(e, "autotune"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / (2.0 * reps);  // per stage launch
    if (ms_per_cfg) ms_per_cfg[c] = per;
    if (per < best_ms) { best_ms = per; best_c = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BSSN_OK) return st;
  if (best) *best = best_c;
  return bssn_batch_set_tile(b, best_c);
}

}  // extern "C"

// ================================================================ server
//
// Continuous batching: a scheduler thread owns a batch.  At every step
// boundary it admits queued requests (in arrival order, skipping any that do
// not fit) while their register bytes fit in the HBM budget and the batch has
// a slot, sets their initial data on the device, advances the resident
// evolutions one RK4 step in one batched graph replay (every one of them, or
// under the shortest-work-first policy the ones with the least work left,
// the others held), and retires the ones
// that reached their step count: their constraint norms are read back, a
// NaN/Inf marks only that request failed, and their registers return to the
// pool.  State stays on the device from admission to retirement.
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t ticket;
  bssn_params p;
  int kind;
  std::vector<double> idp;
  int nsteps;
  double t_submit;
  size_t bytes;
};

struct Res {
  bool done = false;
  bssn_status status = BSSN_EAGAIN;
  double norms[16] = {};
  double latency = 0.0;
  double queued = 0.0;  // seconds from submission to admission
};

struct Act {
  uint64_t ticket;
  int remaining;
  size_t bytes;
  double t_submit;
  long long points;  // interior points
  double t_admit;
  bool held;  // left out of the steps by the shortest-work-first policy
};

}  // namespace

struct bssn_server {
  bssn_batch* batch = nullptr;
  int device = 0;  // the creating thread's device, made current in the scheduler thread
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> queue;
  std::map<uint64_t, Res> results;
  std::map<int, Act> active;
  std::thread th;
  std::atomic<bool> stop{false};
  uint64_t next_ticket = 1;
  // which resident requests a step advances (bssn_server_set_policy)
  int policy = BSSN_SERVE_ALL;
  double min_points = 0.0;
  // statistics
  double t_start = 0.0, busy = 0.0;
  double point_updates = 0.0;
  uint64_t completed = 0, failed = 0;
  std::string error;
};

namespace {

void retire(bssn_server* S, int id, const Act& a) {
  Res r;
  double norms[16];
  bssn_status st = bssn_batch_constraints(S->batch, id, norms);
  bool bad = st != BSSN_OK;
  if (!bad)
    for (int q = 0; q < 16; q++) bad |= !std::isfinite(norms[q]);
  r.done = true;
  r.status = st != BSSN_OK ? st : (bad ? BSSN_EFAILED : BSSN_OK);
  if (st == BSSN_OK) memcpy(r.norms, norms, sizeof(norms));
  r.latency = now_s() - a.t_submit;
  r.queued = a.t_admit - a.t_submit;
  bssn_batch_remove(S->batch, id);
  std::lock_guard<std::mutex> lk(S->mu);
  S->used -= a.bytes;
  S->results[a.ticket] = r;
  S->completed++;
  if (r.status != BSSN_OK) S->failed++;
}

void scheduler(bssn_server* S) {
  // bind the device (and its primary context) to this thread before any other
  // CUDA call: encoding a member's tensor maps is a driver call that needs a
  // current context, and it comes before the first runtime call of an admission
  if (cudaSetDevice(S->device) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->error = "scheduler thread: cudaSetDevice failed";
    S->stop = true;
    return;
  }
  while (!S->stop.load()) {
    // ---- admit at the step boundary
    std::vector<Req> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->active.empty() && S->queue.empty()) {
        S->cv.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      size_t free_b = S->budget - S->used;
      int slots = BSSN_BATCH_MAX_MEMBERS - (int)S->active.size();
      for (auto it = S->queue.begin(); it != S->queue.end() && slots > 0;) {
        if (it->bytes <= free_b) {
          free_b -= it->bytes;
          S->used += it->bytes;
          slots--;
          admit.push_back(std::move(*it));
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (Req& r : admit) {
      int32_t id = -1;
      bssn_status st = bssn_batch_add(S->batch, &r.p, &id);
      if (st == BSSN_OK)
        st = bssn_batch_set_initial_data(S->batch, id, r.kind, r.idp.data(), (int32_t)r.idp.size());
      if (st != BSSN_OK) {
        if (id >= 0) bssn_batch_remove(S->batch, id);
        std::lock_guard<std::mutex> lk(S->mu);
        S->used -= r.bytes;
        // pool fragmented: retry at a later boundary, once a resident request
        // has retired; with none resident the pool is empty and a retry would
        // fail the same way, so the request fails instead
        if (st == BSSN_ENOMEM && !S->active.empty()) {
          S->queue.push_front(std::move(r));
        } else {
          Res res;
          res.done = true;
          res.status = st;
          res.latency = now_s() - r.t_submit;
          S->results[r.ticket] = res;
          S->completed++;
          S->failed++;
        }
        continue;
      }
      Act a{r.ticket, r.nsteps, r.bytes, r.t_submit,
            (long long)r.p.n[0] * r.p.n[1] * r.p.n[2], now_s(), false};
      if (a.remaining <= 0) {
        retire(S, id, a);
        continue;
      }
      std::lock_guard<std::mutex> lk(S->mu);
      S->active[id] = a;
    }
    std::vector<std::pair<int, Act>> done;
    std::vector<std::pair<int, bool>> holds;  // members whose hold changes
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->active.empty()) continue;
      // shortest remaining work first: advance the resident requests with the
      // least work left (steps x interior points) until they hold min_points
      // interior points; the others stay resident and wait
      const int n = (int)S->active.size();
      std::vector<double> work(n), pts(n);
      std::vector<int32_t> sel(n, 1);
      int i = 0;
      for (auto& kv : S->active) {
        work[i] = (double)kv.second.remaining * (double)kv.second.points;
        pts[i] = (double)kv.second.points;
        i++;
      }
      if (S->policy == BSSN_SERVE_SHORTEST) bssn_serve_select(n, work.data(), pts.data(), S->min_points, sel.data());
      i = 0;
      for (auto& kv : S->active) {
        const bool h = sel[i++] == 0;
        if (h != kv.second.held) {
          kv.second.held = h;
          holds.emplace_back(kv.first, h);
        }
      }
    }
    for (auto& hc : holds) bssn_batch_hold(S->batch, hc.first, hc.second ? 1 : 0);
    // ---- one RK4 step for every resident evolution
    const double t0 = now_s();
    bssn_status st = bssn_batch_step(S->batch, 1);
    cudaError_t e = cudaStreamSynchronize(S->batch->stream);
    const double t1 = now_s();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->busy += t1 - t0;
      if (st != BSSN_OK || e != cudaSuccess) {
        S->error = st != BSSN_OK ? std::string("batch step failed") : cudaGetErrorString(e);
        S->stop = true;
        break;
      }
      for (auto it = S->active.begin(); it != S->active.end();) {
        if (it->second.held) {
          ++it;
          continue;
        }
        S->point_updates += (double)it->second.points;
        if (--it->second.remaining <= 0) {
          done.push_back(*it);
          it = S->active.erase(it);
        } else {
          ++it;
        }
      }
    }
    for (auto& d : done) retire(S, d.first, d.second);
  }
}

}  // namespace

extern "C" {

bssn_status bssn_server_create(int32_t precision, size_t hbm_budget_bytes, void* d_pool,
                               size_t pool_bytes, void* cuda_stream, bssn_server** out) {
  if (!out) return bfail(BSSN_EINVAL, "out is NULL");
  *out = nullptr;
  bssn_batch* b = nullptr;
  bssn_status st = bssn_batch_create(precision, BSSN_BATCH_MAX_MEMBERS, d_pool, pool_bytes,
                                     cuda_stream, &b);
  if (st != BSSN_OK) return st;
  bssn_server* S = new (std::nothrow) bssn_server();
  if (!S) {
    bssn_batch_free(b);
    return bfail(BSSN_ENOMEM, "host allocation failed");
  }
  S->batch = b;
  if (cudaGetDevice(&S->device) != cudaSuccess) S->device = 0;
  const size_t cap = pool_bytes - bssn_batch_table_bytes(BSSN_BATCH_MAX_MEMBERS);
  S->budget = std::min(hbm_budget_bytes, cap);
  S->t_start = now_s();
  S->th = std::thread(scheduler, S);
  *out = S;
  return BSSN_OK;
}

bssn_status bssn_submit(bssn_server* S, const bssn_params* p, int32_t id_kind, const double* id_p,
                        int32_t np, int32_t nsteps, uint64_t* ticket) {
  if (!S || !p || !ticket || nsteps < 0 || np < 0 || (np > 0 && !id_p) || np > 33)
    return bfail(BSSN_EINVAL, "bad argument");
  const size_t bytes = bssn_batch_member_bytes(p);
  if (bytes == 0) return BSSN_EINVAL;  // message set by validation
  if (p->precision != S->batch->precision) return bfail(BSSN_EINVAL, "request precision differs from the server's");
  if (bytes > S->budget)
    return bfail(BSSN_EINVAL, "request needs " + std::to_string(bytes) + " bytes, more than the whole budget");
  Req r;
  r.p = *p;
  r.kind = id_kind;
  r.idp.assign(id_p, id_p + np);
  r.nsteps = nsteps;
  r.t_submit = now_s();
  r.bytes = bytes;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop.load()) return bfail(BSSN_EFAILED, "server stopped: " + S->error);
    r.ticket = S->next_ticket++;
    S->results[r.ticket] = Res();
    *ticket = r.ticket;
    S->queue.push_back(std::move(r));
  }
  S->cv.notify_one();
  return BSSN_OK;
}

bssn_status bssn_poll(bssn_server* S, uint64_t ticket, double norms_out[16], double* latency_s) {
  if (!S) return bfail(BSSN_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->results.find(ticket);
  if (it == S->results.end()) return bfail(BSSN_ENOTFOUND, "unknown ticket");
  if (!it->second.done) {
    if (S->stop.load()) return bfail(BSSN_EFAILED, "server stopped: " + S->error);
    return BSSN_EAGAIN;
  }
  if (norms_out) memcpy(norms_out, it->second.norms, sizeof(it->second.norms));
  if (latency_s) *latency_s = it->second.latency;
  return it->second.status;
}

bssn_status bssn_server_set_policy(bssn_server* S, int32_t policy, double min_points) {
  if (!S) return bfail(BSSN_EINVAL, "server is NULL");
  if (policy != BSSN_SERVE_ALL && policy != BSSN_SERVE_SHORTEST) return bfail(BSSN_EINVAL, "unknown policy");
  if (!(min_points >= 0.0)) return bfail(BSSN_EINVAL, "min_points must be >= 0");
  std::lock_guard<std::mutex> lk(S->mu);
  S->policy = policy;
  S->min_points = min_points;
  return BSSN_OK;
}

bssn_status bssn_poll_detail(bssn_server* S, uint64_t ticket, double out[3]) {
  if (!S || !out) return bfail(BSSN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->results.find(ticket);
  if (it == S->results.end()) return bfail(BSSN_ENOTFOUND, "unknown ticket");
  if (!it->second.done) {
    if (S->stop.load()) return bfail(BSSN_EFAILED, "server stopped: " + S->error);
    return BSSN_EAGAIN;
  }
  out[0] = it->second.latency;
  out[1] = it->second.queued;
  out[2] = it->second.latency - it->second.queued;
  return it->second.status;
}

/* out: [0] completed, [1] failed, [2] queued, [3] resident, [4] interior
 * point-updates, [5] busy seconds, [6] wall seconds since create, [7] bytes in use */
bssn_status bssn_server_stats(bssn_server* S, double out[8]) {
  if (!S || !out) return bfail(BSSN_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = (double)S->completed;
  out[1] = (double)S->failed;
  out[2] = (double)S->queue.size();
  out[3] = (double)S->active.size();
  out[4] = S->point_updates;
  out[5] = S->busy;
  out[6] = now_s() - S->t_start;
  out[7] = (double)S->used;
  return BSSN_OK;
}

bssn_status bssn_server_destroy(bssn_server* S) {
  if (!S) return bfail(BSSN_EINVAL, "server is NULL");
  S->stop = true;
  S->cv.notify_all();
  if (S->th.joinable()) S->th.join();
  bssn_status st = bssn_batch_free(S->batch);
  delete S;
  return st;
}

}  // extern "C"
