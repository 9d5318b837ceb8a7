// C ABI of libbssn (include/bssn.h): parameter validation, binding of
// caller-owned device memory, launch sequencing of the RK4 method of lines,
// constraint norms and host<->device state transfer.  No allocation of
// device memory happens here; registers and tables are carved from the block
// given to bssn_alloc.
#include <cmath>
#include <math.h>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bssn_internal.cuh"

using namespace bssn;

namespace {

thread_local std::string g_last_error;

bssn_status fail(bssn_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

bssn_status cuda_fail(cudaError_t e, const char* where) {
  return fail(BSSN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

constexpr size_t ALIGN = 256;
size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

bool validate(const bssn_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return false; }
  for (int d = 0; d < 3; d++)
    if (p->n[d] < 4 || p->n[d] > 4096) { why = "n[d] must be in [4, 4096]"; return false; }
  if (p->ghost != BSSN_GHOST) { why = "ghost must be 3"; return false; }
  if (!(p->h > 0.0) || !std::isfinite(p->h)) { why = "h must be positive and finite"; return false; }
  for (int d = 0; d < 3; d++)
    if (!std::isfinite(p->xmin[d])) { why = "xmin must be finite"; return false; }
  if (p->boundary != BSSN_BC_PERIODIC && p->boundary != BSSN_BC_SOMMERFELD) { why = "bad boundary"; return false; }
  if (p->conformal != BSSN_PHI && p->conformal != BSSN_W) { why = "bad conformal"; return false; }
  if (p->slicing < BSSN_1PLUSLOG || p->slicing > BSSN_GEODESIC) { why = "bad slicing"; return false; }
  if (p->shift != BSSN_GAMMA_DRIVER && p->shift != BSSN_SHIFT_FROZEN) { why = "bad shift"; return false; }
  if (p->precision != BSSN_FP64 && p->precision != BSSN_MIXED && p->precision != BSSN_FF) {
    why = "bad precision";
    return false;
  }
  if (p->ksum_fp64 != 0 && (p->ksum_fp64 != 1 || p->precision != BSSN_MIXED)) {
    why = "ksum_fp64 must be 0, or 1 with mixed precision";
    return false;
  }
  if (!(p->w_fp64_threshold >= 0.0) || !std::isfinite(p->w_fp64_threshold)) {
    why = "w_fp64_threshold must be finite and >= 0";
    return false;
  }
  if (!std::isfinite(p->dt) || !std::isfinite(p->ko_eps) || !std::isfinite(p->eta)) {
    why = "dt, ko_eps and eta must be finite";
    return false;
  }
  if (!(p->w_floor > 0.0)) { why = "w_floor must be positive"; return false; }
  return true;
}

Grid make_grid(const bssn_params* p) {
  Grid g{};
  g.n0 = p->n[0];
  g.n1 = p->n[1];
  g.n2 = p->n[2];
  g.sx = g.n0 + 2 * GH;
  g.sy = g.n1 + 2 * GH;
  g.sz = g.n2 + 2 * GH;
  g.pitch = (g.sx + 7) / 8 * 8;
  g.plane = g.pitch * g.sy;
  g.fstride = g.plane * g.sz;
  g.xmin0 = p->xmin[0];
  g.xmin1 = p->xmin[1];
  g.xmin2 = p->xmin[2];
  g.h = p->h;
  g.periodic = p->boundary == BSSN_BC_PERIODIC;
  g.use_w = p->conformal == BSSN_W;
  g.slicing = p->slicing;
  g.shift = p->shift;
  g.eta = p->eta;
  g.q_R = p->q_R;
  g.ko_eps = p->ko_eps;
  g.w_floor = p->w_floor;
  grid_constants(g);
  return g;
}

// Device block layout.  float64: y_n, k-sum, s1, s2 (+ anchor buffer for
// Sommerfeld).  mixed: y_n in float64 (advanced in place); three float stage
// buffers m[0..2] (m[0] is the float shadow of y_n), each with a float64 W
// array; the float k-sum with its float64 W; float anchors; the derivative
// register of the split stage (135 float fields).
struct Carve {
  size_t reg, yn, ks, s1, s2, ksh, part, out16, err, trk, total, gtab;
  size_t m32[3], mw[3], ks32, ksw, dr, ks64;
  size_t f2[3];  // double-word path: stage buffers of float2 {hi, lo}
  int nblocks;
};

Carve carve(const bssn_params* p, const Grid& g) {
  Carve c{};
  const size_t regb = align_up((size_t)NF * (size_t)g.fstride * sizeof(double));
  const size_t reg32 = align_up((size_t)NF * (size_t)g.fstride * sizeof(float));
  const size_t wb = align_up((size_t)g.fstride * sizeof(double));
  c.reg = regb;
  size_t o = 0;
  c.yn = o; o += regb;
  if (p->precision == BSSN_FP64) {
    c.ks = o; o += regb;
    c.s1 = o; o += regb;
    c.s2 = o; o += regb;
    c.ksh = o;
    if (p->boundary == BSSN_BC_SOMMERFELD) {
      o += regb;
      c.gtab = o;  // ghost-point geometry of the Sommerfeld boundary
      o += align_up(ghost_table_size(g));
    }
  } else if (p->precision == BSSN_FF) {
    // y_n and the k-sum in float64; three double-word stage buffers (s0 the
    // shadow of y_n), each the size of a float64 register; double-word anchors
    c.ks = o; o += regb;
    for (int q = 0; q < 3; q++) {
      c.f2[q] = o; o += regb;
    }
    c.ksh = o;
    if (p->boundary == BSSN_BC_SOMMERFELD) o += regb;
  } else {
    for (int q = 0; q < 3; q++) {
      c.m32[q] = o; o += reg32;
      c.mw[q] = o; o += wb;
    }
    c.ks32 = o; o += reg32;
    c.ksw = o; o += wb;
    if (p->ksum_fp64) {  // the k-sum of every field in float64
      c.ks64 = o; o += regb;
    }
    c.ksh = o;
    if (p->boundary == BSSN_BC_SOMMERFELD) o += reg32;
    c.dr = o; o += align_up((size_t)split_slot_count() * (size_t)g.fstride * sizeof(float));
  }
  c.nblocks = constraints_blocks(g);
  c.part = o; o += align_up((size_t)c.nblocks * 18 * sizeof(double));
  c.out16 = o; o += align_up(16 * sizeof(double));
  c.err = o; o += align_up(sizeof(int));
  c.trk = o; o += align_up(8 * 4 * sizeof(double));
  c.total = o;
  return c;
}

}  // namespace

void bssn::set_last_error(const std::string& msg) { g_last_error = msg; }
bool bssn::validate_params(const bssn_params* p, std::string& why) { return validate(p, why); }
Grid bssn::grid_of(const bssn_params* p) { return make_grid(p); }

struct bssn_ctx {
  bssn_params p;
  Grid g;
  Carve c;
  cudaStream_t stream;
  char* mem;
  double* yn;
  double* ks;
  double* s1;
  double* s2;
  double* ksh;
  void* gtab;  // float64 Sommerfeld: ghost-point geometry table (null otherwise)
  float* m32[3];
  double* mw[3];
  float* ks32;
  double* ksw;
  float* ksh32;
  float* dr;  // mixed: derivative register of the split stage
  double* ks64;  // mixed with ksum_fp64: float64 k-sum of every field (else null)
  float2* f2[3];  // double-word path: stage buffers (f2[0]: shadow of y_n)
  float2* kshf;   // double-word path: boundary anchors
  bool shadow_valid;
  int tile;  // stage-kernel tile configuration (see bssn_autotune)
  CUtensorMap tmap[2][3];  // mixed: tensor maps of the float stage buffers, per TMA box (tma_map)
  bool tmap_ok;
  int* err;             // device error word (bounded waits that gave up)
  int stall_polls;      // test hook of the TMA-staged kernels (bssn_test_stall_tma)
  double* part;
  double* out16;
  double t;
  int npunct;
  double punct[8][4];    // host copy of the punctures {m, x, y, z}
  double* trk;           // device copy, moved by the tracker
  bool tracking;         // advance trk by one Euler step per RK4 step
  bool trk_stale;        // host copy older than trk
  // launch timing (bssn_profile): event pairs around stage and boundary launches
  bool prof;
  std::vector<cudaEvent_t> ev_stage, ev_bc;
  // asynchronous state read-back (bssn_get_state_async): a copy stream, the
  // event after the repack into the read-back area, the event after the copy
  // to the host, and whether that copy may still be running
  cudaStream_t cstream;
  cudaEvent_t ev_out_ready, ev_out_done;
  bool out_pending;
  // caller-owned staging areas for the host copies (bssn_set_staging): the
  // upload and read-back areas in the unpadded host layout, used by no
  // kernel of a step, so that both copies overlap the steps; an upload
  // stream; events: upload landed, upload area free again, read-back area
  // free again (each recorded at least once when the flag is set)
  double* stg_in;
  double* stg_out;
  cudaStream_t istream;
  cudaEvent_t ev_in_ready, ev_in_free, ev_out_free;
  bool in_used, out_used;
};

// Tile configuration indices: [0, tile_config_count()) fused kernels, then
// N_TMA TMA-staged mixed kernels (variant 0: 32x4x1, two blocks per SM;
// 1: 32x8x1, one block per SM; 2: 32x8x1 staging beta^i too), then the
// split-stage variants.
constexpr int N_TMA = 3;
static int tma_variant(int cfg) {
  const int v = cfg - tile_config_count();
  return (v >= 0 && v < N_TMA) ? v : -1;
}
// tensor map of a TMA variant: variants 1 and 2 share the 32x8x1 box
static int tma_map(int v) { return v >= 1 ? 1 : 0; }
static int split_variant(int cfg) {
  const int v = cfg - tile_config_count() - N_TMA;
  return (v >= 0 && v < split_config_count()) ? v : -1;
}
// then the double-word configurations
static int ff_cfg_index(int v) { return tile_config_count() + N_TMA + split_config_count() + v; }
static int ff_variant(int cfg) {
  const int v = cfg - ff_cfg_index(0);
  return (v >= 0 && v < ff_config_count()) ? v : -1;
}

namespace {
cudaError_t prof_mark(bssn_ctx* ctx, std::vector<cudaEvent_t>& v) {
  cudaEvent_t e;
  cudaError_t r = cudaEventCreate(&e);
  if (r != cudaSuccess) return r;
  v.push_back(e);
  return cudaEventRecord(e, ctx->stream);
}
void prof_clear(bssn_ctx* ctx) {
  for (auto e : ctx->ev_stage) cudaEventDestroy(e);
  for (auto e : ctx->ev_bc) cudaEventDestroy(e);
  ctx->ev_stage.clear();
  ctx->ev_bc.clear();
}
}  // namespace

extern "C" {

const char* bssn_last_error(void) { return g_last_error.c_str(); }

bssn_status bssn_layout_of(const bssn_params* p, bssn_layout* out) {
  std::string why;
  if (!out) return fail(BSSN_EINVAL, "out is NULL");
  if (!validate(p, why)) return fail(BSSN_EINVAL, why);
  Grid g = make_grid(p);
  out->stored[0] = g.sx;
  out->stored[1] = g.sy;
  out->stored[2] = g.sz;
  out->ghost = GH;
  out->pitch = g.pitch;
  out->plane = g.plane;
  out->field_stride = g.fstride;
  out->register_elems = (int64_t)NF * g.fstride;
  return BSSN_OK;
}

size_t bssn_required_bytes(const bssn_params* p) {
  std::string why;
  if (!validate(p, why)) {
    g_last_error = why;
    return 0;
  }
  Grid g = make_grid(p);
  return carve(p, g).total;
}

bssn_status bssn_alloc(const bssn_params* p, void* d_mem, size_t bytes, void* cuda_stream,
                       bssn_ctx** out) {
  std::string why;
  if (!out) return fail(BSSN_EINVAL, "out is NULL");
  *out = nullptr;
  if (!validate(p, why)) return fail(BSSN_EINVAL, why);
  if (!d_mem) return fail(BSSN_EINVAL, "d_mem is NULL");
  if (((uintptr_t)d_mem) % ALIGN) return fail(BSSN_EINVAL, "d_mem must be 256-byte aligned");
  Grid g = make_grid(p);
  Carve c = carve(p, g);
  if (bytes < c.total)
    return fail(BSSN_ENOMEM, "memory block too small: need " + std::to_string(c.total) +
                                 " bytes, got " + std::to_string(bytes));
  bssn_ctx* ctx = new (std::nothrow) bssn_ctx();
  if (!ctx) return fail(BSSN_ENOMEM, "host allocation failed");
  ctx->p = *p;
  ctx->g = g;
  ctx->c = c;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->mem = (char*)d_mem;
  ctx->yn = (double*)(ctx->mem + c.yn);
  ctx->ks = p->precision != BSSN_MIXED ? (double*)(ctx->mem + c.ks) : nullptr;
  ctx->s1 = p->precision == BSSN_FP64 ? (double*)(ctx->mem + c.s1) : nullptr;
  ctx->s2 = p->precision == BSSN_FP64 ? (double*)(ctx->mem + c.s2) : nullptr;
  const bool som = p->boundary == BSSN_BC_SOMMERFELD;
  ctx->gtab = nullptr;
  if (p->precision == BSSN_FP64) {
    ctx->ksh = som ? (double*)(ctx->mem + c.ksh) : nullptr;
    ctx->gtab = som ? (void*)(ctx->mem + c.gtab) : nullptr;
  } else if (p->precision == BSSN_FF) {
    for (int q = 0; q < 3; q++) ctx->f2[q] = (float2*)(ctx->mem + c.f2[q]);
    ctx->kshf = som ? (float2*)(ctx->mem + c.ksh) : nullptr;
  } else {
    for (int q = 0; q < 3; q++) {
      ctx->m32[q] = (float*)(ctx->mem + c.m32[q]);
      ctx->mw[q] = (double*)(ctx->mem + c.mw[q]);
    }
    ctx->ks32 = (float*)(ctx->mem + c.ks32);
    ctx->ksw = (double*)(ctx->mem + c.ksw);
    ctx->ksh32 = som ? (float*)(ctx->mem + c.ksh) : nullptr;
    ctx->dr = (float*)(ctx->mem + c.dr);
    ctx->ks64 = p->ksum_fp64 ? (double*)(ctx->mem + c.ks64) : nullptr;
  }
  ctx->shadow_valid = false;
  ctx->tile = p->precision == BSSN_FF ? ff_cfg_index(0) : 0;
  ctx->part = (double*)(ctx->mem + c.part);
  ctx->out16 = (double*)(ctx->mem + c.out16);
  ctx->t = 0.0;
  ctx->npunct = 0;
  ctx->prof = false;
  ctx->err = (int*)(ctx->mem + c.err);
  ctx->stall_polls = 0;
  ctx->trk = (double*)(ctx->mem + c.trk);
  ctx->tracking = false;
  ctx->trk_stale = false;
  ctx->tmap_ok = false;
  if (p->precision == BSSN_MIXED) {
    bool ok = true;
    for (int v = 0; v < 2 && ok; v++)
      for (int q = 0; q < 3 && ok; q++) ok = make_stage_tensor_map(g, ctx->m32[q], &ctx->tmap[v][q], v) == cudaSuccess;
    ctx->tmap_ok = ok;
  }
  ctx->cstream = ctx->istream = nullptr;
  ctx->ev_out_ready = ctx->ev_out_done = ctx->ev_in_ready = ctx->ev_in_free = ctx->ev_out_free = nullptr;
  ctx->out_pending = false;
  ctx->stg_in = ctx->stg_out = nullptr;
  ctx->in_used = ctx->out_used = false;
  if (cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->istream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out_ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in_ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in_free, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out_free, cudaEventDisableTiming) != cudaSuccess ||
      cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream) != cudaSuccess ||
      (ctx->gtab && launch_ghost_table(g, ctx->gtab, ctx->stream) != cudaSuccess)) {
    for (cudaEvent_t ev : {ctx->ev_out_ready, ctx->ev_out_done, ctx->ev_in_ready, ctx->ev_in_free, ctx->ev_out_free})
      if (ev) cudaEventDestroy(ev);
    if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
    if (ctx->istream) cudaStreamDestroy(ctx->istream);
    delete ctx;
    return fail(BSSN_ECUDA, "stream, events or error word init");
  }
  *out = ctx;
  return BSSN_OK;
}

// Work on the library stream that may overwrite the read-back area first
// waits (on the device) for a pending asynchronous copy out of it.
static cudaError_t drain_out(bssn_ctx* ctx) {
  if (!ctx->out_pending) return cudaSuccess;
  ctx->out_pending = false;
  return cudaStreamWaitEvent(ctx->stream, ctx->ev_out_done, 0);
}

bssn_status bssn_free(bssn_ctx* ctx) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  cudaError_t e2 = cudaStreamSynchronize(ctx->cstream);
  cudaError_t e3 = cudaStreamSynchronize(ctx->istream);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = e3;
  prof_clear(ctx);
  for (cudaEvent_t ev : {ctx->ev_out_ready, ctx->ev_out_done, ctx->ev_in_ready, ctx->ev_in_free, ctx->ev_out_free})
    cudaEventDestroy(ev);
  cudaStreamDestroy(ctx->cstream);
  cudaStreamDestroy(ctx->istream);
  delete ctx;
  if (e != cudaSuccess) return cuda_fail(e, "bssn_free");
  return BSSN_OK;
}

bssn_status bssn_state_ptr(bssn_ctx* ctx, double** d_state) {
  if (!ctx || !d_state) return fail(BSSN_EINVAL, "NULL argument");
  *d_state = ctx->yn;
  return BSSN_OK;
}

// Puncture positions: the host copy ctx->punct and the device copy ctx->trk
// that the tracker moves.  push: host -> device (the copy from pageable
// memory is staged before cudaMemcpyAsync returns); pull: device -> host when
// the tracker has run since the last pull.
static cudaError_t push_punct(bssn_ctx* ctx) {
  ctx->trk_stale = false;
  return cudaMemcpyAsync(ctx->trk, &ctx->punct[0][0], sizeof(ctx->punct), cudaMemcpyHostToDevice, ctx->stream);
}
static cudaError_t pull_punct(bssn_ctx* ctx) {
  if (!ctx->trk_stale) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(&ctx->punct[0][0], ctx->trk, sizeof(ctx->punct), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) ctx->trk_stale = false;
  return e;
}

bssn_status bssn_set_initial_data(bssn_ctx* ctx, int32_t kind, const double* p, int32_t np) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  if (np < 0 || (np > 0 && !p)) return fail(BSSN_EINVAL, "bad parameter array");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  double buf[33] = {0};
  int npunct = 0;
  if (kind == BSSN_ID_FLAT) {
  } else if (kind == BSSN_ID_GAUGE_WAVE) {
    if (np < 2) return fail(BSSN_EINVAL, "gauge wave needs {A, d}");
    if (!(p[1] != 0.0) || !(std::fabs(p[0]) < 1.0)) return fail(BSSN_EINVAL, "gauge wave: need |A| < 1, d != 0");
  } else if (kind == BSSN_ID_BL) {
    if (np < 1) return fail(BSSN_EINVAL, "BL needs {npunct, m, x, y, z, ...}");
    npunct = (int)p[0];
    if (npunct < 1 || npunct > 8 || (double)npunct != p[0] || np < 1 + 4 * npunct)
      return fail(BSSN_EINVAL, "BL: npunct must be 1..8 with 4 values each");
  } else if (kind == BSSN_ID_KASNER) {
    if (np < 1 || !(p[0] > 0.0)) return fail(BSSN_EINVAL, "Kasner needs {t0 > 0}");
  } else {
    return fail(BSSN_EINVAL, "unknown initial-data kind");
  }
  const int n = np < 33 ? np : 33;
  for (int q = 0; q < n; q++) buf[q] = p[q];
  cudaError_t e = launch_initial_data(ctx->g, kind, buf, n, ctx->yn, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "initial data");
  ctx->shadow_valid = false;
  ctx->npunct = npunct;
  for (int a = 0; a < npunct; a++)
    for (int q = 0; q < 4; q++) ctx->punct[a][q] = p[1 + 4 * a + q];
  if ((e = push_punct(ctx)) != cudaSuccess) return cuda_fail(e, "punctures");
  ctx->t = 0.0;
  return BSSN_OK;
}

bssn_status bssn_set_adm(bssn_ctx* ctx, const double* host_adm, double t) {
  if (!ctx || !host_adm) return fail(BSSN_EINVAL, "NULL argument");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  const Grid& g = ctx->g;
  cudaError_t e = cudaMemcpy2DAsync(ctx->yn, (size_t)g.pitch * sizeof(double), host_adm,
                                    (size_t)g.sx * sizeof(double), (size_t)g.sx * sizeof(double),
                                    (size_t)16 * g.sz * g.sy, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_adm_to_bssn(g, ctx->yn, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_adm");
  ctx->t = t;
  ctx->shadow_valid = false;
  return BSSN_OK;
}

bssn_status bssn_set_punctures(bssn_ctx* ctx, const double* p, int32_t npunct) {
  if (!ctx || npunct < 0 || npunct > 8 || (npunct > 0 && !p))
    return fail(BSSN_EINVAL, "npunct must be 0..8 with 4 values {m, x, y, z} each");
  ctx->npunct = npunct;
  for (int a = 0; a < npunct; a++)
    for (int q = 0; q < 4; q++) ctx->punct[a][q] = p[4 * a + q];
  cudaError_t e = push_punct(ctx);
  if (e != cudaSuccess) return cuda_fail(e, "punctures");
  return BSSN_OK;
}

bssn_status bssn_set_matter(bssn_ctx* ctx, const double* d_tmunu) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  if (((uintptr_t)d_tmunu) % sizeof(double)) return fail(BSSN_EINVAL, "d_tmunu must be 8-byte aligned");
  ctx->g.tmunu = d_tmunu;
  return BSSN_OK;
}

bssn_status bssn_track_punctures(bssn_ctx* ctx, int32_t enable) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  if (enable && !ctx->tracking && !ctx->trk_stale) {
    cudaError_t e = push_punct(ctx);
    if (e != cudaSuccess) return cuda_fail(e, "punctures");
  }
  ctx->tracking = enable != 0;
  return BSSN_OK;
}

bssn_status bssn_get_punctures(bssn_ctx* ctx, double* out, int32_t* npunct) {
  if (!ctx || !out || !npunct) return fail(BSSN_EINVAL, "NULL argument");
  cudaError_t e = pull_punct(ctx);
  if (e != cudaSuccess) return cuda_fail(e, "punctures");
  *npunct = ctx->npunct;
  for (int a = 0; a < ctx->npunct; a++)
    for (int q = 0; q < 4; q++) out[4 * a + q] = ctx->punct[a][q];
  return BSSN_OK;
}

bssn_status bssn_rhs(bssn_ctx* ctx, const void* d_state, void* d_rhs) {
  if (!ctx || !d_rhs) return fail(BSSN_EINVAL, "NULL argument");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  const double* src = d_state ? (const double*)d_state : ctx->yn;
  double* out = (double*)d_rhs;
  cudaError_t e;
  if (ctx->g.periodic) {
    e = cudaMemsetAsync(out, 0, (size_t)NF * ctx->g.fstride * sizeof(double), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs memset");
  }
  if (ctx->p.precision == BSSN_FP64) {
    StageArgs a{};
    a.src = src;
    a.rhs = out;
    a.mode = MODE_RHS;
    e = launch_stage_fp64(ctx->g, a, ctx->stream, ctx->tile);
    if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs interior");
    if (!ctx->g.periodic) {
      e = launch_sommerfeld(ctx->g, a, nullptr, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs boundary");
    }
    return BSSN_OK;
  }
  if (ctx->p.precision == BSSN_FF) {
    // double-word copy of the state in stage buffer 2
    e = launch_shadow_ff(ctx->g, src, ctx->f2[2], ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs shadow");
    StageArgsFF a{};
    a.src = ctx->f2[2];
    a.rhs = out;
    a.mode = MODE_RHS;
    e = launch_stage_ff(ctx->g, a, ctx->stream, ff_variant(ctx->tile));
    if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs interior");
    if (!ctx->g.periodic) {
      e = launch_sommerfeld_ff(ctx->g, a, nullptr, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs boundary");
    }
    return BSSN_OK;
  }
  // mixed: float copy of the state (with float64 W) in stage buffer 2
  e = launch_shadow(ctx->g, src, ctx->m32[2], ctx->mw[2], ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs shadow");
  StageArgsMixed a{};
  a.src = ctx->m32[2];
  a.srcw = ctx->mw[2];
  a.rhs = out;
  a.w_thr = ctx->p.w_fp64_threshold;
  a.mode = MODE_RHS;
  a.stall_polls = ctx->stall_polls;
  // the selected stage kernel, TMA-staged included (tmap[2] describes m32[2])
  if (split_variant(ctx->tile) >= 0)
    e = launch_stage_mixed_split(ctx->g, a, ctx->dr, ctx->stream, split_variant(ctx->tile));
  else if (tma_variant(ctx->tile) >= 0)
    e = launch_stage_mixed_tma(ctx->g, a, ctx->tmap[tma_map(tma_variant(ctx->tile))][2], ctx->err, ctx->stream,
                               tma_variant(ctx->tile));
  else
    e = launch_stage_mixed(ctx->g, a, ctx->stream, ctx->tile);
  if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs interior");
  if (!ctx->g.periodic) {
    e = launch_sommerfeld_mixed(ctx->g, a, nullptr, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bssn_rhs boundary");
  }
  return BSSN_OK;
}

static bssn_status run_stage(bssn_ctx* ctx, const double* src, int mode, double* out0,
                             double a_dt, double b_dt) {
  StageArgs a{};
  a.src = src;
  a.src0 = ctx->yn;
  a.yn = ctx->yn;
  a.out0 = out0;
  a.ksum = ctx->ks;
  a.kshell = ctx->ksh;
  a.a_dt = a_dt;
  a.a_dtf = (float)a_dt;
  a.b_dt = b_dt;
  a.mode = mode;
  cudaError_t e;
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_stage)) != cudaSuccess) return cuda_fail(e, "profile");
  e = launch_stage_fp64(ctx->g, a, ctx->stream, ctx->tile);
  if (e != cudaSuccess) return cuda_fail(e, "stage");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_stage)) != cudaSuccess) return cuda_fail(e, "profile");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_bc)) != cudaSuccess) return cuda_fail(e, "profile");
  if (ctx->g.periodic) {
    e = launch_periodic_fill(ctx->g, mode == MODE_LAST ? ctx->yn : out0, ctx->stream);
  } else {
    e = launch_sommerfeld(ctx->g, a, ctx->ksh, ctx->stream, ctx->gtab);
  }
  if (e != cudaSuccess) return cuda_fail(e, "boundary");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_bc)) != cudaSuccess) return cuda_fail(e, "profile");
  return BSSN_OK;
}

// mixed stage: src/out are stage-buffer indices into m32/mw (m[0] = shadow of y_n)
static bssn_status run_stage_mixed(bssn_ctx* ctx, int src, int mode, int out, double a_dt,
                                   double b_dt) {
  StageArgsMixed a{};
  a.src = ctx->m32[src];
  a.srcw = ctx->mw[src];
  a.src0 = ctx->m32[0];
  a.src0w = ctx->mw[0];
  a.yn = ctx->yn;
  a.out0 = ctx->m32[out];
  a.out0w = ctx->mw[out];
  a.ksum = ctx->ks32;
  a.ksumw = ctx->ksw;
  a.ksum64 = ctx->ks64;
  a.kshell = ctx->ksh32;
  a.a_dt = a_dt;
  a.a_dtf = (float)a_dt;
  a.b_dt = b_dt;
  a.w_thr = ctx->p.w_fp64_threshold;
  a.mode = mode;
  a.stall_polls = ctx->stall_polls;
  cudaError_t e;
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_stage)) != cudaSuccess) return cuda_fail(e, "profile");
  if (ctx->ks64)
    e = launch_stage_mixed_ks64(ctx->g, a, ctx->stream);
  else if (tma_variant(ctx->tile) >= 0)
    e = launch_stage_mixed_tma(ctx->g, a, ctx->tmap[tma_map(tma_variant(ctx->tile))][src], ctx->err,
                               ctx->stream, tma_variant(ctx->tile));
  else if (split_variant(ctx->tile) >= 0)
    e = launch_stage_mixed_split(ctx->g, a, ctx->dr, ctx->stream, split_variant(ctx->tile));
  else
    e = launch_stage_mixed(ctx->g, a, ctx->stream, ctx->tile);
  if (e != cudaSuccess) return cuda_fail(e, "stage");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_stage)) != cudaSuccess) return cuda_fail(e, "profile");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_bc)) != cudaSuccess) return cuda_fail(e, "profile");
  if (ctx->g.periodic) {
    e = launch_periodic_fill_mixed(ctx->g, ctx->m32[out], ctx->mw[out], ctx->stream);
    if (e == cudaSuccess && mode == MODE_LAST) e = launch_periodic_fill(ctx->g, ctx->yn, ctx->stream);
  } else {
    e = launch_sommerfeld_mixed(ctx->g, a, ctx->ksh32, ctx->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "boundary");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_bc)) != cudaSuccess) return cuda_fail(e, "profile");
  return BSSN_OK;
}

// double-word stage: src/out are stage-buffer indices into f2 (f2[0] = shadow of y_n)
static bssn_status run_stage_ff(bssn_ctx* ctx, int src, int mode, int out, double a_dt, double b_dt) {
  StageArgsFF a{};
  a.src = ctx->f2[src];
  a.src0 = ctx->f2[0];
  a.yn = ctx->yn;
  a.out0 = ctx->f2[out];
  a.ksum = ctx->ks;
  a.kshell = ctx->kshf;
  a.a_dt = a_dt;
  a.b_dt = b_dt;
  a.a_hi = (float)a_dt;
  a.a_lo = (float)(a_dt - (double)a.a_hi);
  a.mode = mode;
  cudaError_t e;
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_stage)) != cudaSuccess) return cuda_fail(e, "profile");
  e = launch_stage_ff(ctx->g, a, ctx->stream, ff_variant(ctx->tile));
  if (e != cudaSuccess) return cuda_fail(e, "stage");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_stage)) != cudaSuccess) return cuda_fail(e, "profile");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_bc)) != cudaSuccess) return cuda_fail(e, "profile");
  if (ctx->g.periodic) {
    // the periodic copy moves 8-byte values whatever they hold
    e = launch_periodic_fill(ctx->g, (double*)ctx->f2[out], ctx->stream);
    if (e == cudaSuccess && mode == MODE_LAST) e = launch_periodic_fill(ctx->g, ctx->yn, ctx->stream);
  } else {
    e = launch_sommerfeld_ff(ctx->g, a, ctx->kshf, ctx->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e, "boundary");
  if (ctx->prof && (e = prof_mark(ctx, ctx->ev_bc)) != cudaSuccess) return cuda_fail(e, "profile");
  return BSSN_OK;
}

bssn_status bssn_rk4_step(bssn_ctx* ctx, int32_t nsteps) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(BSSN_EINVAL, "nsteps < 0");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  const double dt = ctx->p.dt;
  const bool mixed = ctx->p.precision == BSSN_MIXED;
  const bool dword = ctx->p.precision == BSSN_FF;
  for (int s = 0; s < nsteps; s++) {
    bssn_status st;
    cudaError_t e;
    if (ctx->tracking && ctx->npunct > 0) {
      // Euler step of the punctures with the shift of y_n, before y_n moves
      e = launch_track(ctx->g, ctx->yn, ctx->trk, ctx->npunct, dt, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "track");
      ctx->trk_stale = true;
    }
    if (ctx->g.periodic && !((mixed || dword) && ctx->shadow_valid)) {
      e = launch_periodic_fill(ctx->g, ctx->yn, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "periodic fill");
    }
    if (dword) {
      if (!ctx->shadow_valid) {
        e = launch_shadow_ff(ctx->g, ctx->yn, ctx->f2[0], ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "shadow");
        ctx->shadow_valid = true;
      }
      if ((st = run_stage_ff(ctx, 0, MODE_FIRST, 1, 0.5 * dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage_ff(ctx, 1, MODE_MID, 2, 0.5 * dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage_ff(ctx, 2, MODE_MID, 1, dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage_ff(ctx, 1, MODE_LAST, 0, 0.0, dt / 6.0)) != BSSN_OK) return st;
    } else if (!mixed) {
      if ((st = run_stage(ctx, ctx->yn, MODE_FIRST, ctx->s1, 0.5 * dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage(ctx, ctx->s1, MODE_MID, ctx->s2, 0.5 * dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage(ctx, ctx->s2, MODE_MID, ctx->s1, dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage(ctx, ctx->s1, MODE_LAST, nullptr, 0.0, dt / 6.0)) != BSSN_OK) return st;
    } else {
      if (!ctx->shadow_valid) {
        e = launch_shadow(ctx->g, ctx->yn, ctx->m32[0], ctx->mw[0], ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "shadow");
        ctx->shadow_valid = true;
      }
      if ((st = run_stage_mixed(ctx, 0, MODE_FIRST, 1, 0.5 * dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage_mixed(ctx, 1, MODE_MID, 2, 0.5 * dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage_mixed(ctx, 2, MODE_MID, 1, dt, 0.0)) != BSSN_OK) return st;
      if ((st = run_stage_mixed(ctx, 1, MODE_LAST, 0, 0.0, dt / 6.0)) != BSSN_OK) return st;
    }
    ctx->t += dt;
  }
  return BSSN_OK;
}

static bssn_status check_err(bssn_ctx* ctx);

// Scratch for the 12 ADM fields of the analysis kernels: a stage buffer that
// holds nothing between RK4 steps (float64: s1; mixed: the float stage buffer
// m[1], 24 floats = 12 doubles per point).  Stream order keeps a following
// step from overwriting it early.
static double* adm_scratch(bssn_ctx* ctx) {
  if (ctx->p.precision == BSSN_FF) return (double*)ctx->f2[1];
  return ctx->p.precision == BSSN_FP64 ? ctx->s1 : (double*)ctx->m32[1];
}

bssn_status bssn_constraints(bssn_ctx* ctx, double out[16]) {
  if (!ctx || !out) return fail(BSSN_EINVAL, "NULL argument");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  if (bssn_status es = check_err(ctx)) return es;
  cudaError_t e = pull_punct(ctx);
  if (e != cudaSuccess) return cuda_fail(e, "punctures");
  e = launch_constraints(ctx->g, ctx->yn, &ctx->punct[0][0], ctx->npunct,
                                     ctx->p.r_excise, ctx->part, ctx->c.nblocks, ctx->out16,
                                     ctx->stream, adm_scratch(ctx));
  if (e != cudaSuccess) return cuda_fail(e, "constraints");
  e = cudaMemcpyAsync(out, ctx->out16, 16 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "constraints copy");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "constraints sync");
  return BSSN_OK;
}

bssn_status bssn_adm_integrals(bssn_ctx* ctx, double* d_dens, double out[8]) {
  if (!ctx || !out) return fail(BSSN_EINVAL, "NULL argument");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  if (bssn_status es = check_err(ctx)) return es;
  cudaError_t e = pull_punct(ctx);
  if (e != cudaSuccess) return cuda_fail(e, "punctures");
  Punct pu{};
  pu.n = ctx->npunct;
  for (int a = 0; a < pu.n; a++)
    for (int q = 0; q < 4; q++) pu.p[a][q] = ctx->punct[a][q];
  pu.r_ex = ctx->p.r_excise;
  e = launch_adm_integrals(ctx->g, ctx->yn, pu, d_dens, ctx->part, adm_integrals_blocks(ctx->g), ctx->out16,
                           ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "adm integrals");
  e = cudaMemcpyAsync(out, ctx->out16, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "adm integrals copy");
  return BSSN_OK;
}

bssn_status bssn_psi4(bssn_ctx* ctx, double* d_out) {
  if (!ctx || !d_out) return fail(BSSN_EINVAL, "NULL argument");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  cudaError_t e = launch_psi4(ctx->g, ctx->yn, d_out, ctx->stream, adm_scratch(ctx));
  if (e != cudaSuccess) return cuda_fail(e, "psi4");
  return BSSN_OK;
}

// Read and clear the device error word (a bounded wait in a kernel gave up).
static bssn_status check_err(bssn_ctx* ctx) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "error word");
  if (h) {
    cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream);
    return fail(BSSN_ETIMEOUT, "a stage kernel gave up waiting for its shared-memory tile; the state is invalid");
  }
  return BSSN_OK;
}

// Staging area for the host copies of the state: a stage buffer that holds
// nothing between RK4 steps (float64: s1, 24 fields; mixed: the float stage
// buffer m[1], 12 fields of doubles).  Host copies are contiguous blocks of
// whole fields, repacked into the pitched layout on the device.
static double* stage_area(bssn_ctx* ctx, int* fields) {
  if (ctx->p.precision == BSSN_FP64) {
    *fields = NF;
    return ctx->s1;
  }
  if (ctx->p.precision == BSSN_FF) {  // a double-word register holds 24 fields of doubles
    *fields = NF;
    return (double*)ctx->f2[1];
  }
  *fields = NF / 2;
  return (double*)ctx->m32[1];
}

// shadow: uploads also write the mixed path's float shadow of y_n
static cudaError_t copy_state(bssn_ctx* ctx, double* host, bool to_device, bool shadow = false) {
  const Grid& g = ctx->g;
  const size_t per = (size_t)g.sx * g.sy * g.sz;
  int chunk = 0;
  double* area = stage_area(ctx, &chunk);
  cudaError_t e = cudaSuccess;
  float* s32 = shadow ? ctx->m32[0] : nullptr;
  double* w = shadow ? ctx->mw[0] : nullptr;
  for (int f0 = 0; f0 < NF && e == cudaSuccess; f0 += chunk) {
    const int nf = f0 + chunk <= NF ? chunk : NF - f0;
    const size_t bytes = per * nf * sizeof(double);
    if (to_device) {
      e = cudaMemcpyAsync(area, host + per * f0, bytes, cudaMemcpyHostToDevice, ctx->stream);
      if (e == cudaSuccess) e = launch_repack(g, area, ctx->yn, f0, nf, true, ctx->stream, s32, w);
    } else {
      e = launch_repack(g, area, ctx->yn, f0, nf, false, ctx->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(host + per * f0, area, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    }
  }
  return e;
}

// Read-back area of bssn_get_state_async, disjoint from the staging area of
// the uploads (so that a copy out and the next upload can run at the same
// time): float64: s2; mixed: the float buffers m[2] and m[0] (12 fields of
// doubles each; m[0], the float shadow of y_n, is rebuilt before the next
// step).  Returns the number of areas (1 or 2) and their field counts.
static int out_areas(bssn_ctx* ctx, double* area[2], int nf[2]) {
  if (ctx->p.precision == BSSN_FP64) {
    area[0] = ctx->s2;
    nf[0] = NF;
    return 1;
  }
  if (ctx->p.precision == BSSN_FF) {
    area[0] = (double*)ctx->f2[2];
    nf[0] = NF;
    return 1;
  }
  area[0] = (double*)ctx->m32[2];
  area[1] = (double*)ctx->m32[0];
  nf[0] = nf[1] = NF / 2;
  return 2;
}

bssn_status bssn_get_state(bssn_ctx* ctx, double* host, double* t) {
  if (!ctx || !host) return fail(BSSN_EINVAL, "NULL argument");
  if (bssn_status es = check_err(ctx)) return es;
  cudaError_t e = drain_out(ctx);
  if (e == cudaSuccess) e = copy_state(ctx, host, false);
  if (e != cudaSuccess) return cuda_fail(e, "get_state copy");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_state sync");
  if (t) *t = ctx->t;
  return BSSN_OK;
}

bssn_status bssn_set_state(bssn_ctx* ctx, const double* host, double t) {
  bssn_status st = bssn_set_state_async(ctx, host, t);
  if (st != BSSN_OK) return st;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_state sync");
  return BSSN_OK;
}

// Bytes of one staging area: the state in the unpadded host layout.
static size_t stage_copy_bytes(const Grid& g) { return (size_t)NF * g.sx * g.sy * g.sz * sizeof(double); }

bssn_status bssn_set_state_async(bssn_ctx* ctx, const double* host, double t) {
  if (!ctx || !host) return fail(BSSN_EINVAL, "NULL argument");
  cudaError_t e = cudaSuccess;
  // the repack also forms the mixed path's float shadow of y_n, unless a copy
  // out of the shadow buffer (the read-back area without staging) may still
  // run, or the grid is periodic (the next step refreshes the ghosts of y_n
  // first and forms the shadow from them)
  const bool shadow = ctx->p.precision == BSSN_MIXED && !ctx->out_pending && !ctx->g.periodic;
  float* s32 = shadow ? ctx->m32[0] : nullptr;
  double* w = shadow ? ctx->mw[0] : nullptr;
  if (ctx->stg_in) {
    // upload on the upload stream, into the staging area, while the library
    // stream may still be stepping; then repacked into y_n in stream order
    if (ctx->in_used) e = cudaStreamWaitEvent(ctx->istream, ctx->ev_in_free, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->stg_in, host, stage_copy_bytes(ctx->g), cudaMemcpyHostToDevice, ctx->istream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_in_ready, ctx->istream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_in_ready, 0);
    if (e == cudaSuccess) e = launch_repack(ctx->g, ctx->stg_in, ctx->yn, 0, NF, true, ctx->stream, s32, w);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_in_free, ctx->stream);
    if (e == cudaSuccess) ctx->in_used = true;
  } else {
    e = copy_state(ctx, const_cast<double*>(host), true, shadow);
  }
  if (e != cudaSuccess) return cuda_fail(e, "set_state copy");
  ctx->t = t;
  ctx->shadow_valid = shadow;
  return BSSN_OK;
}

size_t bssn_staging_bytes(const bssn_params* p) {
  std::string why;
  if (!validate(p, why)) {
    fail(BSSN_EINVAL, why);
    return 0;
  }
  return 2 * align_up(stage_copy_bytes(make_grid(p)));
}

bssn_status bssn_set_staging(bssn_ctx* ctx, void* d_mem, size_t bytes) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->cstream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->istream);
  if (e != cudaSuccess) return cuda_fail(e, "set_staging sync");
  ctx->in_used = ctx->out_used = false;
  if (!d_mem) {
    ctx->stg_in = ctx->stg_out = nullptr;
    return BSSN_OK;
  }
  const size_t area = align_up(stage_copy_bytes(ctx->g));
  if (((uintptr_t)d_mem) % ALIGN) return fail(BSSN_EINVAL, "d_mem must be 256-byte aligned");
  if (bytes < 2 * area)
    return fail(BSSN_ENOMEM, "staging block too small: need " + std::to_string(2 * area) + " bytes");
  ctx->stg_in = (double*)d_mem;
  ctx->stg_out = (double*)((char*)d_mem + area);
  return BSSN_OK;
}

bssn_status bssn_get_state_async(bssn_ctx* ctx, double* host, double* t) {
  if (!ctx || !host) return fail(BSSN_EINVAL, "NULL argument");
  if (ctx->stg_out) {
    // repack into the caller's read-back area (free once the previous copy
    // out of it is done), copied to the host on the copy stream
    cudaError_t e = ctx->out_used ? cudaStreamWaitEvent(ctx->stream, ctx->ev_out_free, 0) : cudaSuccess;
    if (e == cudaSuccess) e = launch_repack(ctx->g, ctx->stg_out, ctx->yn, 0, NF, false, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out_ready, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cstream, ctx->ev_out_ready, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host, ctx->stg_out, stage_copy_bytes(ctx->g), cudaMemcpyDeviceToHost, ctx->cstream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out_free, ctx->cstream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state_async");
    ctx->out_used = true;
    if (t) *t = ctx->t;
    return BSSN_OK;
  }
  const Grid& g = ctx->g;
  const size_t per = (size_t)g.sx * g.sy * g.sz;
  double* area[2];
  int nf[2];
  const int na = out_areas(ctx, area, nf);
  cudaError_t e = drain_out(ctx);  // the previous copy out of these areas is done
  for (int q = 0, f0 = 0; q < na && e == cudaSuccess; f0 += nf[q], q++)
    e = launch_repack(g, area[q], ctx->yn, f0, nf[q], false, ctx->stream);
  if (ctx->p.precision == BSSN_MIXED) ctx->shadow_valid = false;
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out_ready, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cstream, ctx->ev_out_ready, 0);
  for (int q = 0, f0 = 0; q < na && e == cudaSuccess; f0 += nf[q], q++)
    e = cudaMemcpyAsync(host + per * f0, area[q], per * nf[q] * sizeof(double), cudaMemcpyDeviceToHost,
                        ctx->cstream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out_done, ctx->cstream);
  if (e != cudaSuccess) return cuda_fail(e, "get_state_async");
  ctx->out_pending = true;
  if (t) *t = ctx->t;
  return BSSN_OK;
}

bssn_status bssn_wait_state(bssn_ctx* ctx) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  cudaError_t e2 = cudaStreamSynchronize(ctx->cstream);
  cudaError_t e3 = cudaStreamSynchronize(ctx->istream);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) return cuda_fail(e, "wait_state");
  return check_err(ctx);
}

// Configurations: [0, tile_config_count()) the fused kernels; the next
// N_TMA the TMA-staged mixed kernels; then the split-stage
// variants.
int32_t bssn_tile_count(void) { return tile_config_count() + N_TMA + split_config_count() + ff_config_count(); }

const char* bssn_tile_name(int32_t cfg) {
  if (ff_variant(cfg) >= 0) return ff_config_name(ff_variant(cfg));
  if (tma_variant(cfg) == 0) return "tma32x4x1/2";
  if (tma_variant(cfg) == 1) return "tma32x8x1/1";
  if (tma_variant(cfg) == 2) return "tma11_32x8x1/1";
  if (split_variant(cfg) >= 0) return split_config_name(split_variant(cfg));
  return tile_config_name(cfg);
}

static bool tile_usable(const bssn_ctx* ctx, int cfg) {
  if (cfg < 0 || cfg >= bssn_tile_count()) return false;
  if ((ff_variant(cfg) >= 0) != (ctx->p.precision == BSSN_FF)) return false;
  if (cfg < tile_config_count() && ctx->p.precision == BSSN_FP64 && !tile_config_has_fp64(cfg)) return false;
  if (tma_variant(cfg) >= 0) return ctx->p.precision == BSSN_MIXED && ctx->tmap_ok;
  if (split_variant(cfg) >= 0) return ctx->p.precision == BSSN_MIXED;
  return true;
}

bssn_status bssn_set_tile(bssn_ctx* ctx, int32_t cfg) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  if (!tile_usable(ctx, cfg))
    return fail(BSSN_EINVAL,
                "tile config out of range or not for this precision (the TMA and split kernels are for the "
                "mixed path, the ff kernels for the double-word path)");
  ctx->tile = cfg;
  return BSSN_OK;
}

bssn_status bssn_autotune(bssn_ctx* ctx, int32_t reps, int32_t* best, double* ms_per_cfg) {
  if (!ctx || reps < 1) return fail(BSSN_EINVAL, "bad argument");
  if (cudaError_t ed = drain_out(ctx)) return cuda_fail(ed, "wait for the state read-back");
  const bool mixed = ctx->p.precision == BSSN_MIXED;
  const bool dword = ctx->p.precision == BSSN_FF;
  if ((mixed || dword) && !ctx->shadow_valid) {
    cudaError_t e = mixed ? launch_shadow(ctx->g, ctx->yn, ctx->m32[0], ctx->mw[0], ctx->stream)
                          : launch_shadow_ff(ctx->g, ctx->yn, ctx->f2[0], ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "shadow");
    ctx->shadow_valid = true;
  }
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e, "event");
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(e, "event"); }
  const int ncfg = bssn_tile_count();
  double best_ms = 1e300;
  int best_c = 0;
  bssn_status st = BSSN_OK;
  // Each repetition times the first two stages (first: y_n -> stage buffer 1
  // and k-sum; second: stage buffer 1 -> stage buffer 2, k-sum accumulated),
  // which leave y_n (and its float shadow) unchanged; the next step
  // overwrites what they wrote.  The second stage carries the combine's extra
  // loads, which the first alone would not weigh.
  for (int c = 0; c < ncfg && st == BSSN_OK; c++) {
    if (!tile_usable(ctx, c)) {
      if (ms_per_cfg) ms_per_cfg[c] = INFINITY;
      continue;
    }
    auto launch1 = [&](int stage) -> cudaError_t {
      const bool second = stage == 1;
      if (dword) {
        StageArgsFF a{};
        a.src = ctx->f2[second ? 1 : 0]; a.src0 = ctx->f2[0]; a.yn = ctx->yn;
        a.out0 = ctx->f2[second ? 2 : 1]; a.ksum = ctx->ks; a.a_dt = 0.5 * ctx->p.dt;
        a.a_hi = (float)a.a_dt; a.a_lo = (float)(a.a_dt - (double)a.a_hi);
        a.mode = second ? MODE_MID : MODE_FIRST;
        return launch_stage_ff(ctx->g, a, ctx->stream, ff_variant(c));
      }
      if (!mixed) {
        StageArgs a{};
        a.src = second ? ctx->s1 : ctx->yn; a.src0 = ctx->yn; a.yn = ctx->yn;
        a.out0 = second ? ctx->s2 : ctx->s1; a.ksum = ctx->ks;
        a.a_dt = 0.5 * ctx->p.dt; a.mode = second ? MODE_MID : MODE_FIRST;
        return launch_stage_fp64(ctx->g, a, ctx->stream, c);
      }
      const int q = second ? 1 : 0, o = second ? 2 : 1;
      StageArgsMixed a{};
      a.src = ctx->m32[q]; a.srcw = ctx->mw[q]; a.src0 = ctx->m32[0]; a.src0w = ctx->mw[0];
      a.yn = ctx->yn; a.out0 = ctx->m32[o]; a.out0w = ctx->mw[o];
      a.ksum = ctx->ks32; a.ksumw = ctx->ksw; a.ksum64 = ctx->ks64; a.a_dt = 0.5 * ctx->p.dt;
      a.a_dtf = (float)a.a_dt;
      a.w_thr = ctx->p.w_fp64_threshold; a.mode = second ? MODE_MID : MODE_FIRST;
      if (ctx->ks64) return launch_stage_mixed_ks64(ctx->g, a, ctx->stream);
      if (tma_variant(c) >= 0)
        return launch_stage_mixed_tma(ctx->g, a, ctx->tmap[tma_map(tma_variant(c))][q], ctx->err, ctx->stream,
                                      tma_variant(c));
      if (split_variant(c) >= 0)
        return launch_stage_mixed_split(ctx->g, a, ctx->dr, ctx->stream, split_variant(c));
      return launch_stage_mixed(ctx->g, a, ctx->stream, c);
    };
    auto launch = [&]() -> cudaError_t {
      cudaError_t r = launch1(0);
      return r == cudaSuccess ? launch1(1) : r;
    };
    if ((e = launch()) != cudaSuccess) { st = cuda_fail(e, "autotune warm-up"); break; }
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < reps && e == cudaSuccess; r++) e = launch();
    cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { st = cuda_fail(e, "autotune"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / (2.0 * reps);  // per stage launch
    if (ms_per_cfg) ms_per_cfg[c] = per;
    if (per < best_ms) { best_ms = per; best_c = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BSSN_OK) return st;
  ctx->tile = best_c;
  if (best) *best = best_c;
  return BSSN_OK;
}

bssn_status bssn_test_stall_tma(bssn_ctx* ctx, int32_t polls) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  if (polls < 0 || polls > (1 << 20)) return fail(BSSN_EINVAL, "polls must be in [0, 2^20]");
  ctx->stall_polls = polls;
  return BSSN_OK;
}

bssn_status bssn_profile(bssn_ctx* ctx, int32_t enable, double out[4]) {
  if (!ctx) return fail(BSSN_EINVAL, "ctx is NULL");
  if (enable) {
    prof_clear(ctx);
    ctx->prof = true;
    return BSSN_OK;
  }
  ctx->prof = false;
  if (!out) return fail(BSSN_EINVAL, "out is NULL");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "profile sync");
  std::vector<cudaEvent_t>* lists[2] = {&ctx->ev_stage, &ctx->ev_bc};
  for (int q = 0; q < 2; q++) {
    double ms = 0.0;
    const auto& v = *lists[q];
    for (size_t i = 0; i + 1 < v.size(); i += 2) {
      float x = 0.f;
      e = cudaEventElapsedTime(&x, v[i], v[i + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "profile elapsed");
      ms += x;
    }
    out[2 * q] = ms;
    out[2 * q + 1] = (double)(v.size() / 2);
  }
  prof_clear(ctx);
  return BSSN_OK;
}

}  // extern "C"
