// bssn_constraints_noalloc: constraint norms for callers that cannot hand the
// library a device memory block.
//
// Who needs this: a host program that owns every device allocation itself
// (an arena that reserved all of HBM up front, a plug-in host that forbids
// its plug-ins to allocate, a real-time loop that may not call cudaMalloc
// because cudaMalloc can synchronise the device and stall other work) but
// still wants the Hamiltonian/momentum norms of a state buffer it holds.
// The regular entry point (bssn_constraints) carves its reduction scratch out
// of the block given to bssn_alloc; this one keeps that scratch in a fixed
// static device array instead, so it allocates nothing.
//
// The per-block partial sums live in a file-scope __device__ array of
// NOALLOC_MAX_BLOCKS x 18 doubles (2.25 MiB), loaded into every GPU that loads
// the library and kept until the process exits.  That bounds the grid to
// BSSN_NOALLOC_MAX_POINTS interior points; larger grids are rejected.
//
// In host code the array's name is only a host-side stand-in, so its device
// address is resolved with cudaGetSymbolAddress, once per device, with that
// device current, on the first call made on that device.
#include <cmath>
#include <mutex>
#include <string>

#include "bssn_internal.cuh"

namespace bssn {
namespace {

constexpr int NOALLOC_MAX_BLOCKS = BSSN_NOALLOC_MAX_POINTS / 256;
constexpr int NOALLOC_PART = 18;  // partials per block (as in k_constraints.cu)
constexpr int MAX_DEVICES = 64;

// Shared by every call on a device: the last call's partials stay here.  Every
// entry a call reads is written earlier in the same call, so nothing has to
// start at zero; calls that overlap on the GPU race on this memory.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * NOALLOC_PART];
static __device__ __align__(256) double g_noalloc_out[16];

struct SymbolAddrs {
  double* partials = nullptr;
  double* out = nullptr;
  bool done = false;
};
SymbolAddrs g_addrs[MAX_DEVICES];
std::mutex g_addrs_mu;

// Resolve the device addresses of the static arrays on the current device.
// Only a successful lookup is remembered: after a failure (for instance a
// first call made while the stream was being captured) the next call looks
// the addresses up again.
cudaError_t resolve(int dev, double** partials, double** out) {
  std::lock_guard<std::mutex> lk(g_addrs_mu);
  SymbolAddrs& s = g_addrs[dev];
  if (!s.done) {
    void* p = nullptr;
    void* o = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&o, g_noalloc_out);
    if (e != cudaSuccess) return e;
    s.partials = (double*)p;
    s.out = (double*)o;
    s.done = true;
  }
  *partials = s.partials;
  *out = s.out;
  return cudaSuccess;
}

bssn_status nfail(bssn_status st, const std::string& m) {
  set_last_error(m);
  return st;
}

}  // namespace
}  // namespace bssn

using namespace bssn;

extern "C" bssn_status bssn_constraints_noalloc(const bssn_params* p, const double* d_state,
                                                const double* punct, int32_t npunct,
                                                void* cuda_stream, double out[16]) {
  bssn_layout lay;
  if (!p || !d_state || !out) return nfail(BSSN_EINVAL, "NULL argument");
  if (bssn_layout_of(p, &lay) != BSSN_OK) return BSSN_EINVAL;  // message set by bssn_layout_of
  if (npunct < 0 || npunct > 8 || (npunct > 0 && !punct))
    return nfail(BSSN_EINVAL, "npunct must be 0..8 with 4 values each");
  const long long pts = (long long)p->n[0] * p->n[1] * p->n[2];
  if (pts > BSSN_NOALLOC_MAX_POINTS)
    return nfail(BSSN_EINVAL, "bssn_constraints_noalloc: grid has " + std::to_string(pts) +
                                  " interior points, the static scratch holds at most " +
                                  std::to_string((long long)BSSN_NOALLOC_MAX_POINTS) +
                                  "; use bssn_constraints with a bssn_alloc context");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(BSSN_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return nfail(BSSN_EINVAL, "device ordinal out of range");
  double* partials = nullptr;
  double* dout = nullptr;
  e = resolve(dev, &partials, &dout);
  if (e != cudaSuccess)
    return nfail(BSSN_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

  // The same grid description the context-based path builds.
  const Grid g = grid_of(p);
  const int nblocks = constraints_blocks(g);
  if (nblocks > NOALLOC_MAX_BLOCKS) return nfail(BSSN_EINVAL, "grid too large for the static scratch");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  e = launch_constraints(g, d_state, punct, npunct, p->r_excise, partials, nblocks, dout, s);
  if (e != cudaSuccess) return nfail(BSSN_ECUDA, std::string("constraints: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(out, dout, 16 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return nfail(BSSN_ECUDA, std::string("copy: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return nfail(BSSN_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
  return BSSN_OK;
}
