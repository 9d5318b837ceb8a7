// Outer boundary: Sommerfeld radiative condition (arXiv:1111.3344, Sec.
// "Boundary Conditions") and periodic ghost copies.
//
// Sommerfeld: at each ghost point b the radiative part is
//   rad = -v0 (x^i / r) d_i X - v0 (X - X0) / r
// with second-order derivatives (centred where both neighbours are stored,
// one-sided inward on the outermost layer), plus the p = 2 power-law
// correction taken from the inner neighbour j = b - n (n the sum of the
// outward normals of the faces b lies beyond), layer by layer from the
// innermost outwards: rhs_b = rad_b + (r_j / r_b)^2 (rhs_j - rad_j).
// Unrolled along the chain b -> j -> ... -> a (a the first interior point)
// the factors telescope to
//   rhs_b = rad_b + (r_a / r_b)^2 (rhs_a - rad_a),
// so each ghost point is independent: one thread per ghost point, no layer
// ordering.  X0 = 1 for alpha, W and the diagonal of gt, else 0; v0 = sqrt 2
// for alpha and K, else 1.  The boundary arithmetic is float64 on both paths.
#include "boundary_point.cuh"

namespace bssn {

template <bool PRE>
__global__ void sommerfeld_fp64_kernel(Grid g, StageArgs a, const double* __restrict__ kanchor) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ghost_count(g)) return;
  sommerfeld_point_fp64<PRE>(g, a, kanchor, q);
}

// blockIdx.y: one of four field groups (W and gt_ij; K and At_ij but its last;
// the rest of At_ij, Gt^i, alpha; beta^i and B^i)
__global__ void sommerfeld_anchor_fp64_kernel(Grid g, StageArgs a, double* __restrict__ kanchor) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= shell_count(g)) return;
  switch (blockIdx.y) {
    case 0: sommerfeld_anchor_fp64<0, 7>(g, a, kanchor, q); break;
    case 1: sommerfeld_anchor_fp64<7, 13>(g, a, kanchor, q); break;
    case 2: sommerfeld_anchor_fp64<13, 18>(g, a, kanchor, q); break;
    default: sommerfeld_anchor_fp64<18, NF>(g, a, kanchor, q); break;
  }
}

__global__ void sommerfeld_fp64_tab_kernel(Grid g, StageArgs a, const double* __restrict__ kanchor,
                                           const double* __restrict__ tab, const long long* __restrict__ itab) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ghost_count(g)) return;
  switch (blockIdx.y) {  // six groups of four fields
    case 0: sommerfeld_point_fp64_tab<0, 4>(g, a, kanchor, tab, itab, q); break;
    case 1: sommerfeld_point_fp64_tab<4, 8>(g, a, kanchor, tab, itab, q); break;
    case 2: sommerfeld_point_fp64_tab<8, 12>(g, a, kanchor, tab, itab, q); break;
    case 3: sommerfeld_point_fp64_tab<12, 16>(g, a, kanchor, tab, itab, q); break;
    case 4: sommerfeld_point_fp64_tab<16, 20>(g, a, kanchor, tab, itab, q); break;
    default: sommerfeld_point_fp64_tab<20, NF>(g, a, kanchor, tab, itab, q); break;
  }
}

__global__ void ghost_table_kernel(Grid g, double* __restrict__ tab, long long* __restrict__ itab) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ghost_count(g)) return;
  ghost_table_fill(g, q, tab, itab);
}

cudaError_t launch_ghost_table(const Grid& g, void* table, cudaStream_t s) {
  const unsigned total = ghost_count(g);
  double* tab = (double*)table;
  long long* itab = (long long*)(tab + (size_t)GEO_DOUBLES * total);
  ghost_table_kernel<<<(total + 127) / 128, 128, 0, s>>>(g, tab, itab);
  return cudaGetLastError();
}
size_t ghost_table_size(const Grid& g) { return ghost_table_bytes(g); }

// one thread per ghost point, every field (geometry formed once)
// mixed: blockIdx.y picks one of four field groups (W and gt_ij; K and
// At_ij but its last; the rest of At_ij, Gt^i, alpha; beta^i and B^i), each
// a few unrolled fields per thread (their loads in flight together; the
// kernel is bound by load latency)
__global__ void sommerfeld_mixed_kernel(Grid g, StageArgsMixed a, const float* __restrict__ kanchor) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ghost_count(g)) return;
  switch (blockIdx.y) {
    case 0: sommerfeld_point_mixed_fields<0, 7, true>(g, a, kanchor, q); break;
    case 1: sommerfeld_point_mixed_fields<7, 13, true>(g, a, kanchor, q); break;
    case 2: sommerfeld_point_mixed_fields<13, 18, true>(g, a, kanchor, q); break;
    default: sommerfeld_point_mixed_fields<18, NF, true>(g, a, kanchor, q); break;
  }
}

template <typename S>
__global__ void periodic_fill_kernel(Grid g, S* __restrict__ y, double* __restrict__ w) {
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ghost_count(g)) return;
  periodic_point<S>(g, y, w, q);
}

// Stage modes: the anchor pass (one thread per shell point) turns the k left at
// the anchors into k - rad once, then the ghost points each form only their
// own radiative term.  MODE_RHS (no anchors): every ghost point forms both.
cudaError_t launch_sommerfeld(const Grid& g, const StageArgs& a, const double* kanchor,
                              cudaStream_t s, const void* table) {
  const unsigned total = ghost_count(g);
  const int bs = 128;
  if (a.mode != MODE_RHS && kanchor) {
    const unsigned ns = shell_count(g);
    sommerfeld_anchor_fp64_kernel<<<dim3((ns + bs - 1) / bs, 4), bs, 0, s>>>(g, a, const_cast<double*>(kanchor));
    if (table) {
      const double* tab = (const double*)table;
      const long long* itab = (const long long*)(tab + (size_t)GEO_DOUBLES * total);
      sommerfeld_fp64_tab_kernel<<<dim3((total + bs - 1) / bs, 6), bs, 0, s>>>(g, a, kanchor, tab, itab);
    } else {
      sommerfeld_fp64_kernel<true><<<(total + bs - 1) / bs, bs, 0, s>>>(g, a, kanchor);
    }
  } else {
    sommerfeld_fp64_kernel<false><<<(total + bs - 1) / bs, bs, 0, s>>>(g, a, kanchor);
  }
  return cudaGetLastError();
}
cudaError_t launch_sommerfeld_mixed(const Grid& g, const StageArgsMixed& a, const float* kanchor,
                                    cudaStream_t s) {
  const unsigned total = ghost_count(g);
  const int bs = 128;
  sommerfeld_mixed_kernel<<<dim3((total + bs - 1) / bs, 4), bs, 0, s>>>(g, a, kanchor);
  return cudaGetLastError();
}

cudaError_t launch_periodic_fill(const Grid& g, double* y, cudaStream_t s) {
  const unsigned total = ghost_count(g);
  periodic_fill_kernel<double><<<(total + 255) / 256, 256, 0, s>>>(g, y, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_periodic_fill_mixed(const Grid& g, float* y, double* w, cudaStream_t s) {
  const unsigned total = ghost_count(g);
  periodic_fill_kernel<float><<<(total + 255) / 256, 256, 0, s>>>(g, y, w);
  return cudaGetLastError();
}

// Repacking between the unpadded host layout (nf fields of sz x sy x sx
// doubles, contiguous) and the pitched register layout, fields f0 .. f0+nf-1:
// the host copies then move one contiguous block at full link speed.
// Host-layout <-> register repacking: fields f0 .. f0+nf-1, every stored
// point; the host layout has no x padding.  One warp-row of a block per stored
// row of one field (consecutive x, coalesced on both sides), rows grid-strided:
// no per-element index division.  Unpacking can also write the float shadow
// of y_n (X - X0, the mixed path's stage input) and its float64 W.
constexpr int RP_X = 32, RP_Y = 8;

__global__ void __launch_bounds__(RP_X * RP_Y)
    unpack_fields_kernel(Grid g, const double* __restrict__ flat, double* __restrict__ reg, int f0, int nf,
                         float* __restrict__ s32, double* __restrict__ w) {
  const long long rows = (long long)g.sy * g.sz;
  const long long total = rows * nf;
  for (long long r = (long long)blockIdx.x * RP_Y + threadIdx.y; r < total; r += (long long)gridDim.x * RP_Y) {
    const int f = (int)(r / rows);
    const long long rr = r - f * rows;  // k sy + j
    const double* src = flat + r * g.sx;
    const long long o = (long long)(f0 + f) * g.fstride + rr * g.pitch;
    const double bg = background(g, f0 + f);
    for (int i = threadIdx.x; i < g.sx; i += RP_X) {
      const double v = src[i];
      reg[o + i] = v;
      if (s32) {
        s32[o + i] = (float)(v - bg);
        if (f0 + f == F_CHI) w[rr * g.pitch + i] = v;
      }
    }
  }
}

__global__ void __launch_bounds__(RP_X * RP_Y)
    pack_fields_kernel(Grid g, const double* __restrict__ reg, double* __restrict__ flat, int f0, int nf) {
  const long long rows = (long long)g.sy * g.sz;
  const long long total = rows * nf;
  for (long long r = (long long)blockIdx.x * RP_Y + threadIdx.y; r < total; r += (long long)gridDim.x * RP_Y) {
    const int f = (int)(r / rows);
    const long long rr = r - f * rows;
    double* dst = flat + r * g.sx;
    const long long o = (long long)(f0 + f) * g.fstride + rr * g.pitch;
    for (int i = threadIdx.x; i < g.sx; i += RP_X) dst[i] = reg[o + i];
  }
}

cudaError_t launch_repack(const Grid& g, double* flat, double* reg, int f0, int nf, bool to_reg, cudaStream_t s,
                          float* s32, double* w) {
  const dim3 block(RP_X, RP_Y), grid(152 * 16);
  if (to_reg) unpack_fields_kernel<<<grid, block, 0, s>>>(g, flat, reg, f0, nf, s32, w);
  else pack_fields_kernel<<<grid, block, 0, s>>>(g, reg, flat, f0, nf);
  return cudaGetLastError();
}

}  // namespace bssn
