// Internal definitions shared by the CUDA translation units of libbssn.
// Not part of the public ABI (include/bssn.h is).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bssn.h"

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
};

__host__ __device__ inline long long lin(const Grid& g, int i, int j, int k) {
  return (long long)k * g.plane + (long long)j * g.pitch + i;
}

// RK4 stage combination modes of the fused stage kernel.
enum StageMode : int {
  MODE_RHS = 0,     // rhs <- k
  MODE_FIRST = 1,   // out0 <- yn + a dt k ; acc <- yn + b dt k
  MODE_MID = 2,     // out0 <- yn + a dt k ; acc <- acc + b dt k
  MODE_LAST = 3,    // acc <- acc + b dt k ; out0 <- acc (mixed: float shadow of y_{n+1})
};

// Arguments of a fused stage.  S is the storage type of the stage buffers:
// double on the float64 path; float on the mixed path, where every stage
// buffer also carries W (field 0) in float64 in a separate array (w suffix).
template <typename S>
struct StageArgsT {
  const S* src;          // stage input state (stencil source)
  const double* srcw;    // mixed: float64 W of the stage input (else null)
  const double* yn;      // y_n (float64)
  S* out0;               // next stage state (FIRST/MID); mixed LAST: shadow of y_{n+1}
  double* out0w;         // mixed: float64 W of out0 (else null)
  double* acc;           // accumulator (float64)
  double* rhs;           // MODE_RHS output (float64 register)
  S* kshell;             // if non-null: k at interior points next to the outer boundary
  double a_dt, b_dt;     // stage coefficients times dt
  double w_thr;          // mixed: W below this -> W right-hand side in float64
  int mode;
};
using StageArgs = StageArgsT<double>;
using StageArgsMixed = StageArgsT<float>;

// Launch wrappers (defined in the .cu files); all return cudaError_t of the launch.
cudaError_t launch_stage_fp64(const Grid& g, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_mixed(const Grid& g, const StageArgsMixed& a, cudaStream_t s);
cudaError_t launch_sommerfeld(const Grid& g, const StageArgs& a, const double* kanchor,
                              cudaStream_t s);
cudaError_t launch_sommerfeld_mixed(const Grid& g, const StageArgsMixed& a, const float* kanchor,
                                    cudaStream_t s);
cudaError_t launch_periodic_fill(const Grid& g, double* y, cudaStream_t s);
cudaError_t launch_periodic_fill_mixed(const Grid& g, float* y, double* w, cudaStream_t s);
cudaError_t launch_shadow(const Grid& g, const double* y, float* s32, double* w, cudaStream_t s);
cudaError_t launch_initial_data(const Grid& g, int kind, const double* dparams, int np,
                                double* y, cudaStream_t s);
cudaError_t launch_constraints(const Grid& g, const double* y, const double* dpunct,
                               int npunct, double r_excise, double* partials, int nblocks,
                               double* dout16, cudaStream_t s);
int constraints_blocks(const Grid& g);

}  // namespace bssn
