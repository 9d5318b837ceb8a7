// Arithmetic-pipe peaks of the GPU the library runs on: the rates against
// which the float64 and float32 stage kernels are placed on a roofline (the
// stencil path has no tensor-core work, so the peaks that bound it are the
// float64 and float32 FMA pipes and HBM).
//
// Every thread runs CHAINS independent multiply-add chains a = a*x + y for
// ITERS iterations (x slightly below 1 and y small, so the values settle and
// neither overflow nor become subnormal); 152 x 4 blocks of 256 threads keep
// every SM's pipe busy.  A chain result is stored only if it equals a value it
// can never take, so the stores cost nothing and the compiler must still
// compute every chain.  Two flops per multiply-add.
#include <cuda_runtime.h>

#include "bssn_internal.cuh"

namespace bssn {
namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;
constexpr int BLOCKS = 152 * 4;

template <typename T, int ITERS>
__global__ void __launch_bounds__(THREADS) fma_chain_kernel(T x, T y, T* __restrict__ sink) {
  T a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; c++) a[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 4
  for (int it = 0; it < ITERS; it++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) a[c] = fma(a[c], x, y);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CHAINS; c++) s += a[c];
  if (s == T(-1)) sink[0] = s;  // never true: a[c] stays positive
}

template <typename T, int ITERS>
cudaError_t time_chain(void* d_sink, cudaStream_t s, int reps, double* gflops) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  const T x = T(0.999999), y = T(1e-7);
  fma_chain_kernel<T, ITERS><<<BLOCKS, THREADS, 0, s>>>(x, y, (T*)d_sink);  // warm-up
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; r++) {
    fma_chain_kernel<T, ITERS><<<BLOCKS, THREADS, 0, s>>>(x, y, (T*)d_sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double flop = 2.0 * CHAINS * (double)ITERS * THREADS * BLOCKS * reps;
  *gflops = flop / (ms * 1e-3) / 1e9;
  return cudaSuccess;
}

}  // namespace
}  // namespace bssn

using namespace bssn;

extern "C" bssn_status bssn_peak_probe(int32_t kind, void* d_sink, void* cuda_stream, int32_t reps,
                                       double* gflops) {
  if (!d_sink || !gflops || reps < 1 || (kind != 0 && kind != 1)) {
    set_last_error("bssn_peak_probe: kind must be 0 (float64) or 1 (float32), reps >= 1, pointers non-NULL");
    return BSSN_EINVAL;
  }
  if (((uintptr_t)d_sink) % sizeof(double)) {
    set_last_error("bssn_peak_probe: d_sink must be 8-byte aligned");
    return BSSN_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // float64: about 10 GFLOP a launch (some 8 ms on a GB300); float32 the same
  // launch count with 32x the iterations
  const cudaError_t e = kind == 0 ? time_chain<double, 4096>(d_sink, s, reps, gflops)
                                  : time_chain<float, 4096 * 32>(d_sink, s, reps, gflops);
  if (e != cudaSuccess) {
    set_last_error(std::string("bssn_peak_probe: ") + cudaGetErrorString(e));
    return BSSN_ECUDA;
  }
  return BSSN_OK;
}
