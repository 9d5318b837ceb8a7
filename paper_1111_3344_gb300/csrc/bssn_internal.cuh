// Internal definitions shared by the CUDA translation units of libbssn.
// Not part of the public ABI (include/bssn.h is).
#pragma once
#include <atomic>
#include <cstdint>
#include <string>
#include <type_traits>
#include <cuda.h>
#include <cuda_runtime.h>

#include "bssn.h"
#include "ff.cuh"

namespace bssn {

constexpr int NF = BSSN_NUM_FIELDS;  // 24 evolved grid functions
constexpr int GH = 3;                // ghost width

// Field order (same as the ABI): 0 phi|W, 1..6 gt_ij, 7 trK, 8..13 At_ij,
// 14..16 Gt^i, 17 alpha, 18..20 beta^i, 21..23 B^i.
enum : int { F_CHI = 0, F_GT = 1, F_TRK = 7, F_AT = 8, F_GAM = 14, F_ALP = 17, F_BETA = 18, F_B = 21 };

// Symmetric pair index (xx xy xz yy yz zz) and its inverse.
__host__ __device__ constexpr int sym(int a, int b) {
  return a == b ? (a == 0 ? 0 : (a == 1 ? 3 : 5))
                : ((a + b) == 1 ? 1 : ((a + b) == 2 ? 2 : 4));
}

// Grid + method parameters in the form the kernels read (passed by value).
struct Grid {
  int n0, n1, n2;        // interior points per axis
  int sx, sy, sz;        // stored points per axis (n + 2*GH)
  long long pitch;       // elements per stored x-row (>= sx, multiple of 8)
  long long plane;       // pitch * sy
  long long fstride;     // elements per field = plane * sz
  double xmin0, xmin1, xmin2;
  double h;
  int periodic;
  int use_w;
  int slicing;           // BSSN_1PLUSLOG / BSSN_HARMONIC / BSSN_GEODESIC
  int shift;             // BSSN_GAMMA_DRIVER / BSSN_SHIFT_FROZEN
  double eta, q_R;       // q_R <= 0 or inf: q == 1
  double ko_eps;
  double w_floor;
  // stencil and boundary constants, precomputed on the host in both
  // precisions (a float64 division or conversion costs a slot of the slow
  // float64 pipe on every thread that would otherwise compute it)
  double i12h, i12h2, i144h2, kos, i2h;  // 1/(12h), 1/(12h^2), 1/(144h^2), eps/(64h), 1/(2h)
  float i12hf, i12h2f, i144h2f, kosf, i2hf, w_floorf, etaf, hf;
  // the float remainders d - (double)f of the same constants (the low words
  // of their double-word forms)
  float i12hl, i12h2l, i144h2l, kosl, w_floorl, etal;
  float xminf[3];
  // stress-energy tensor T_{mu nu} (10 fields in the register layout: T_00,
  // T_0x, T_0y, T_0z, T_xx, T_xy, T_xz, T_yy, T_yz, T_zz), or null (vacuum)
  const double* tmunu;
};

// Host-side fill of the derived constants of a Grid.
inline void grid_constants(Grid& g) {
  g.i12h = 1.0 / (12.0 * g.h);
  g.i12h2 = 1.0 / (12.0 * g.h * g.h);
  g.i144h2 = 1.0 / (144.0 * g.h * g.h);
  g.kos = g.ko_eps / (64.0 * g.h);
  g.i2h = 0.5 / g.h;
  g.i12hf = (float)g.i12h;
  g.i12h2f = (float)g.i12h2;
  g.i144h2f = (float)g.i144h2;
  g.kosf = (float)g.kos;
  g.i2hf = (float)g.i2h;
  g.w_floorf = (float)g.w_floor;
  g.etaf = (float)g.eta;
  g.hf = (float)g.h;
  g.xminf[0] = (float)g.xmin0;
  g.xminf[1] = (float)g.xmin1;
  g.xminf[2] = (float)g.xmin2;
  g.i12hl = (float)(g.i12h - (double)g.i12hf);
  g.i12h2l = (float)(g.i12h2 - (double)g.i12h2f);
  g.i144h2l = (float)(g.i144h2 - (double)g.i144h2f);
  g.kosl = (float)(g.kos - (double)g.kosf);
  g.w_floorl = (float)(g.w_floor - (double)g.w_floorf);
  g.etal = (float)(g.eta - (double)g.etaf);
}

// Pick the float64, float or double-word (float f + remainder l) copy of a
// constant.
template <typename T>
__host__ __device__ __forceinline__ T gc(double d, float f, float l);
template <>
__host__ __device__ __forceinline__ double gc<double>(double d, float, float) { return d; }
template <>
__host__ __device__ __forceinline__ float gc<float>(double, float f, float) { return f; }
template <>
__host__ __device__ __forceinline__ ff gc<ff>(double, float f, float l) { return ff(f, l); }

// Raise kernel's dynamic shared-memory limit to bytes on the current device,
// once per device: the attribute belongs to the kernel as loaded in that
// device's context.  done holds one bit per device (devices 32 and up set the
// attribute at every call); concurrent callers may both set it, which is
// harmless.
template <typename K>
inline cudaError_t smem_optin(K kernel, int bytes, std::atomic<unsigned>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned bit = dev >= 0 && dev < 32 ? 1u << dev : 0u;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <typename T>
constexpr bool is_f32 = std::is_same<T, float>::value;
template <typename T>
constexpr bool is_f64 = std::is_same<T, double>::value;

// Matter projections of T_{mu nu} at linear index id (Sec. "Spacetime Curvature
// Evolution"): E = (T_00 - 2 beta^i T_0i + beta^i beta^j T_ij)/alpha^2,
// S_i = -(T_0i - beta^j T_ij)/alpha, S_ij = T_ij (6 components), in type T.
template <typename T>
__device__ __forceinline__ void matter_at(const Grid& g, long long id, T alp, const T beta[3], T& E, T Si[3],
                                          T Sij[6]) {
  const double* p = g.tmunu + id;
  const long long fs = g.fstride;
  const T T00 = T(__ldg(p));
  T T0[3];
#pragma unroll
  for (int a = 0; a < 3; a++) T0[a] = T(__ldg(p + (1 + a) * fs));
#pragma unroll
  for (int m = 0; m < 6; m++) Sij[m] = T(__ldg(p + (4 + m) * fs));
  T e = T00;
#pragma unroll
  for (int a = 0; a < 3; a++) e -= T(2) * beta[a] * T0[a];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) e += beta[a] * beta[b] * Sij[sym(a, b)];
  const T ia = T(1) / alp;
  E = e * ia * ia;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    T s = T0[a];
#pragma unroll
    for (int b = 0; b < 3; b++) s -= beta[b] * Sij[sym(b, a)];
    Si[a] = -s * ia;
  }
}

// Coordinate of interior index ii (cell centre), xmin + (ii + 1/2) h, with the
// product and the sum rounded separately (no fused multiply-add), so that a
// coordinate that is exactly 0 comes out as 0 (the z axis of the Psi4 triad)
// and the excision tests see the same values as a plain evaluation.
__device__ __forceinline__ double cell_coord(double xmin, int ii, double h) {
  return __dadd_rn(xmin, __dmul_rn((double)ii + 0.5, h));
}

__host__ __device__ inline long long lin(const Grid& g, int i, int j, int k) {
  return (long long)k * g.plane + (long long)j * g.pitch + i;
}

// Ghost points of a grid, enumerated compactly: the three bottom and three top
// z-slabs (whole planes), then per interior z-plane the three front and three
// back y-rows (whole rows) and the three left and three right points of every
// interior row.  Consecutive indices are mostly consecutive in x.
__host__ __device__ inline unsigned ghost_count(const Grid& g) {
  return 6u * g.sx * g.sy + (unsigned)g.n2 * (6u * g.sx + 6u * g.n1);
}
__host__ __device__ inline void ghost_decode(const Grid& g, unsigned q, int& i, int& j, int& k) {
  const unsigned pl = (unsigned)g.sx * g.sy;
  const unsigned slab = 3u * pl;
  if (q < 2u * slab) {
    const unsigned top = q >= slab;
    const unsigned r = q - top * slab;
    k = (int)(r / pl) + (top ? GH + g.n2 : 0);
    const unsigned rem = r % pl;
    j = (int)(rem / g.sx);
    i = (int)(rem % g.sx);
    return;
  }
  const unsigned per = 6u * g.sx + 6u * g.n1;
  const unsigned q2 = q - 2u * slab;
  k = GH + (int)(q2 / per);
  unsigned r = q2 % per;
  if (r < 3u * g.sx) {
    j = (int)(r / g.sx);
    i = (int)(r % g.sx);
  } else if (r < 6u * g.sx) {
    r -= 3u * g.sx;
    j = GH + g.n1 + (int)(r / g.sx);
    i = (int)(r % g.sx);
  } else {
    r -= 6u * g.sx;
    j = GH + (int)(r / 6u);
    const int c = (int)(r % 6u);
    i = c < GH ? c : GH + g.n0 + (c - GH);
  }
}

// Interior points next to the outer boundary (the anchors of the Sommerfeld
// closed form), enumerated: the bottom and top interior z-planes, then per
// interior z-plane its first and last interior rows, then the first and last
// point of every other row.  Interior indices (0 .. n-1).
__host__ __device__ inline unsigned shell_count(const Grid& g) {
  if (g.n2 < 2) return (unsigned)g.n0 * g.n1 * g.n2;
  const unsigned per = (g.n1 < 2) ? (unsigned)g.n0 : 2u * g.n0 + 2u * (g.n1 - 2);
  return 2u * g.n0 * g.n1 + (unsigned)(g.n2 - 2) * per;
}
__host__ __device__ inline void shell_decode(const Grid& g, unsigned q, int& ii, int& jj, int& kk) {
  const unsigned pl = (unsigned)g.n0 * g.n1;
  if (q < 2u * pl) {
    kk = q < pl ? 0 : g.n2 - 1;
    const unsigned r = q % pl;
    jj = (int)(r / g.n0);
    ii = (int)(r % g.n0);
    return;
  }
  const unsigned per = 2u * g.n0 + 2u * (g.n1 - 2);
  const unsigned q2 = q - 2u * pl;
  kk = 1 + (int)(q2 / per);
  unsigned r = q2 % per;
  if (r < 2u * g.n0) {
    jj = r < (unsigned)g.n0 ? 0 : g.n1 - 1;
    ii = (int)(r % g.n0);
  } else {
    r -= 2u * g.n0;
    jj = 1 + (int)(r / 2u);
    ii = (r & 1u) ? g.n0 - 1 : 0;
  }
}

// RK4 stage combination modes of the fused stage kernel.  Classical RK4 as
//   y_{n+1} = y_n + dt/6 (k1 + 2 k2 + 2 k3 + k4),
// with y_n advanced in place once per step and the weighted sum of the k kept
// in a k-sum register (a, b below already include dt):
//   FIRST  out0 <- base + a k ; ksum <- k          (k = k1, source y_n)
//   MID    out0 <- base + a k ; ksum <- ksum + 2 k  (k2, k3)
//   LAST   yn   <- yn + b (ksum + k)                (k4, b = dt/6)
// base is y_n (float64 path) or the float shadow of y_n (mixed path, where
// LAST also refreshes that shadow into out0).  MODE_RHS writes k to rhs.
enum StageMode : int {
  MODE_RHS = 0,
  MODE_FIRST = 1,
  MODE_MID = 2,
  MODE_LAST = 3,
};

// Arguments of a fused stage.  S is the storage type of the stage buffers:
// double on the float64 path; float on the mixed path, where every stage
// buffer also carries W (field 0) in float64 in a separate array (w suffix)
// and the float fields hold X - X0 (see background()).
template <typename S>
struct StageArgsT {
  const S* src;          // stage input state (stencil source)
  const double* srcw;    // mixed: float64 W of the stage input (else null)
  const S* src0;         // base of the stage values: y_n (float64) / its float shadow (mixed)
  const double* src0w;   // mixed: float64 W of the shadow
  double* yn;            // y_n (float64), advanced in place by LAST
  S* out0;               // next stage state (FIRST/MID); mixed LAST: shadow of y_{n+1}
  double* out0w;         // mixed: float64 W of out0 (else null)
  S* ksum;               // k1 + 2 k2 + 2 k3
  double* ksumw;         // mixed: the same for W in float64
  double* ksum64;        // mixed: if non-null, the k-sum of every field in float64 (ksum unused)
  double* rhs;           // MODE_RHS output (float64 register)
  S* kshell;             // if non-null: k at interior points next to the outer boundary
  double a_dt, b_dt;     // stage coefficients times dt
  float a_dtf;           // a_dt as float (mixed stage values)
  double w_thr;          // mixed: W below this -> W right-hand side in float64
  int mode;
  // test hook of the TMA-staged kernels: > 0 issues no tile copy and gives up
  // waiting after this many polls, so that the bounded-wait path runs with
  // nothing in flight; 0 in normal operation
  int stall_polls;
};
using StageArgs = StageArgsT<double>;
using StageArgsMixed = StageArgsT<float>;

// Arguments of a fused stage of the double-word path: the stage buffers hold
// double-word values (float2 {hi, lo}) of X itself; y_n and the weighted sum
// of the k are float64; the right-hand side runs in double-word arithmetic.
struct StageArgsFF {
  const float2* src;   // stage input (stencil source)
  const float2* src0;  // double-word shadow of y_n (base of the stage values)
  double* yn;          // y_n, advanced in place by LAST
  float2* out0;        // next stage state (FIRST/MID); LAST: the shadow of y_{n+1}
  double* ksum;        // k1 + 2 k2 + 2 k3, float64
  double* rhs;         // MODE_RHS output (float64 register)
  float2* kshell;      // if non-null: k at interior points next to the outer boundary
  double a_dt, b_dt;   // stage coefficients times dt
  float a_hi, a_lo;    // a_dt as a double-word constant
  int mode;
};

// Punctures {m, x, y, z} (at most 8) and the excision radius of the excised
// norms and integrals, passed to kernels by value.
struct Punct {
  double p[8][4];
  int n;
  double r_ex;
};

// Launch wrappers (defined in the .cu files); all return cudaError_t of the launch.
cudaError_t launch_stage_fp64(const Grid& g, const StageArgs& a, cudaStream_t s, int cfg = 0);
cudaError_t launch_stage_mixed(const Grid& g, const StageArgsMixed& a, cudaStream_t s, int cfg = 0);
cudaError_t launch_stage_mixed_ks64(const Grid& g, const StageArgsMixed& a, cudaStream_t s);
int tile_config_count();
bool tile_config_has_fp64(int c);  // false for the mixed-only configurations
const char* tile_config_name(int c);
// TMA-staged mixed stage kernel (k_stage_tma.cu); map describes the float
// stage buffer that is the stencil source.
// Tensor map of a float stage buffer for TMA-staged variant v (0: 32 x 4 x 1
// tiles, 1: 32 x 8 x 1; the box is the tile plus three ghost layers).
cudaError_t make_stage_tensor_map(const Grid& g, const float* base, CUtensorMap* out, int variant = 0);
cudaError_t launch_stage_mixed_tma(const Grid& g, const StageArgsMixed& a, const CUtensorMap& map,
                                   int* err, cudaStream_t s, int variant = 0);
// sets the TMA variant's dynamic shared-memory limit (call outside graph capture)
cudaError_t prepare_stage_mixed_tma(int variant);
// Split mixed stage (k_stage_split.cu): a stencil pass into the derivative
// register dr (split_slot_count() float fields of the register layout) and an
// algebra pass.
int split_slot_count();
int split_config_count();
const char* split_config_name(int v);
cudaError_t launch_stage_mixed_split(const Grid& g, const StageArgsMixed& a, float* dr, cudaStream_t s,
                                     int variant);
// table (may be null): the context's ghost-geometry table (launch_ghost_table)
cudaError_t launch_sommerfeld(const Grid& g, const StageArgs& a, const double* kanchor,
                              cudaStream_t s, const void* table = nullptr);
size_t ghost_table_size(const Grid& g);
cudaError_t launch_ghost_table(const Grid& g, void* table, cudaStream_t s);
cudaError_t launch_sommerfeld_mixed(const Grid& g, const StageArgsMixed& a, const float* kanchor,
                                    cudaStream_t s);
cudaError_t launch_periodic_fill(const Grid& g, double* y, cudaStream_t s);
// Double-word path (k_stage_ff.cu): fused stage in configuration cfg
// (ff_config_count() of them), Sommerfeld boundary (float64 arithmetic on the
// double-word stage values), double-word shadow of a float64 register.
int ff_config_count();
const char* ff_config_name(int c);
cudaError_t launch_stage_ff(const Grid& g, const StageArgsFF& a, cudaStream_t s, int cfg);
cudaError_t launch_sommerfeld_ff(const Grid& g, const StageArgsFF& a, const float2* kanchor, cudaStream_t s);
cudaError_t launch_shadow_ff(const Grid& g, const double* y, float2* s2, cudaStream_t s);
cudaError_t launch_periodic_fill_mixed(const Grid& g, float* y, double* w, cudaStream_t s);
cudaError_t launch_shadow(const Grid& g, const double* y, float* s32, double* w, cudaStream_t s);
// Copy fields f0 .. f0+nf-1 between a contiguous unpadded block flat and the
// pitched register reg (to_reg: flat -> reg) (k_boundary.cu).
// to_reg: host layout -> register, and (s32, w non-null) the float shadow
// X - X0 and float64 W of the mixed path as well
cudaError_t launch_repack(const Grid& g, double* flat, double* reg, int f0, int nf, bool to_reg, cudaStream_t s,
                          float* s32 = nullptr, double* w = nullptr);
cudaError_t launch_initial_data(const Grid& g, int kind, const double* dparams, int np,
                                double* y, cudaStream_t s);
// adm_scratch (may be null): 12 * fstride doubles; when given, the ADM fields
// are formed once per stored point there (launch_adm_fields) instead of at
// every stencil point.
cudaError_t launch_constraints(const Grid& g, const double* y, const double* dpunct,
                               int npunct, double r_excise, double* partials, int nblocks,
                               double* dout16, cudaStream_t s, double* adm_scratch = nullptr);
// gamma_ij and K_ij (12 fields) at every stored point of y (k_constraints.cu).
cudaError_t launch_adm_fields(const Grid& g, const double* y, double* adm, cudaStream_t s);
int constraints_blocks(const Grid& g);
// y's first 16 field slots hold ADM data (alpha, beta^i, gamma_ij, K_ij);
// converts it in place to the BSSN state (k_adm.cu).
cudaError_t launch_adm_to_bssn(const Grid& g, double* y, cudaStream_t s);
// ADM mass / angular momentum integrals (k_adm_integrals.cu): dout8 receives
// M, J_x, J_y, J_z over all interior points then over the excised set; dens
// (4 fields of the register layout, may be null) the integrands.  partials
// holds adm_integrals_blocks(g) * 8 doubles.
int adm_integrals_blocks(const Grid& g);
cudaError_t launch_adm_integrals(const Grid& g, const double* y, const Punct& pu, double* dens,
                                 double* partials, int nblocks, double* dout8, cudaStream_t s);
// Weyl scalar Psi4 at interior points into out (2 fields of the register
// layout: real, imaginary) (k_psi4.cu).
cudaError_t launch_psi4(const Grid& g, const double* y, double* out, cudaStream_t s,
                        double* adm_scratch = nullptr);
// One Euler step of the puncture positions dpunct (rows {m, x, y, z}) from the
// shift of y (k_track.cu).
cudaError_t launch_track(const Grid& g, const double* y, double* dpunct, int np, double dt, cudaStream_t s);

// Sets the message bssn_last_error() returns on the calling thread.
void set_last_error(const std::string& msg);
// Parameter validation and grid description shared by the context and batch paths.
bool validate_params(const bssn_params* p, std::string& why);
Grid grid_of(const bssn_params* p);

}  // namespace bssn
