// Initial data on the device: closed-form BSSN variables of the analytic data
// sets (arXiv:1111.3344, Sec. "Initial Conditions": BSSN quantities from
// their definitions with B^i = 0), one thread per stored point.
//  FLAT        Minkowski.
//  GAUGE_WAVE  H = 1 - A sin(2 pi x / d): alpha = sqrt H, gamma_xx = H, so
//              phi = ln(H)/12, W = H^{-1/6}, gt = diag(H^{2/3}, H^{-1/3},
//              H^{-1/3}), K = H'/(2 H^{3/2}), At = diag(H' H^{-5/6}/3,
//              -H' H^{-11/6}/6, -H' H^{-11/6}/6), Gt^x = (2/3) H' H^{-5/3}.
//  BL          psi = 1 + sum m_a/(2 r_a): W = psi^-2, phi = ln psi, gt = delta,
//              alpha = psi^-2, everything else 0.
//  KASNER(t)   W = t^{-1/3}, phi = ln(t)/6, gt = diag(t^{2/3}, t^{2/3},
//              t^{-4/3}), K = -1/t, At = diag(-t^{-1/3}/3, -t^{-1/3}/3,
//              2 t^{-7/3}/3), alpha = 1 (Sec. "Cosmology").
#include "bssn_internal.cuh"

namespace bssn {

struct IdParams {
  double p[33];
  int np;
};

__global__ void initial_data_kernel(Grid g, int kind, IdParams ip, double* __restrict__ y) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)g.sx * g.sy * g.sz;
  if (tid >= total) return;
  const int i = (int)(tid % g.sx);
  const int j = (int)((tid / g.sx) % g.sy);
  const int k = (int)(tid / ((long long)g.sx * g.sy));
  const double x = g.xmin0 + (i - GH + 0.5) * g.h;
  const double yv = g.xmin1 + (j - GH + 0.5) * g.h;
  const double z = g.xmin2 + (k - GH + 0.5) * g.h;
  double v[NF];
  for (int f = 0; f < NF; f++) v[f] = 0.0;
  v[F_GT + 0] = v[F_GT + 3] = v[F_GT + 5] = 1.0;
  v[F_ALP] = 1.0;
  v[F_CHI] = g.use_w ? 1.0 : 0.0;
  if (kind == BSSN_ID_GAUGE_WAVE) {
    const double A = ip.p[0], d = ip.p[1];
    const double ph = 2.0 * 3.14159265358979323846 * x / d;
    const double H = 1.0 - A * sin(ph);
    const double Hp = -A * (2.0 * 3.14159265358979323846 / d) * cos(ph);
    const double lH = log(H);
    v[F_CHI] = g.use_w ? exp(-lH / 6.0) : lH / 12.0;
    v[F_GT + 0] = exp(lH * (2.0 / 3.0));
    v[F_GT + 3] = v[F_GT + 5] = exp(-lH / 3.0);
    v[F_TRK] = Hp / (2.0 * H * sqrt(H));
    v[F_AT + 0] = Hp * exp(-lH * (5.0 / 6.0)) / 3.0;
    v[F_AT + 3] = v[F_AT + 5] = -Hp * exp(-lH * (11.0 / 6.0)) / 6.0;
    v[F_GAM + 0] = (2.0 / 3.0) * Hp * exp(-lH * (5.0 / 3.0));
    v[F_ALP] = sqrt(H);
  } else if (kind == BSSN_ID_BL) {
    const int n = (int)ip.p[0];
    double psi = 1.0;
    for (int a = 0; a < n; a++) {
      const double* q = ip.p + 1 + 4 * a;
      const double dx = x - q[1], dy = yv - q[2], dz = z - q[3];
      psi += q[0] / (2.0 * sqrt(dx * dx + dy * dy + dz * dz));
    }
    v[F_CHI] = g.use_w ? 1.0 / (psi * psi) : log(psi);
    v[F_ALP] = 1.0 / (psi * psi);
  } else if (kind == BSSN_ID_KASNER) {
    const double t = ip.p[0];
    const double lt = log(t);
    v[F_CHI] = g.use_w ? exp(-lt / 3.0) : lt / 6.0;
    v[F_GT + 0] = v[F_GT + 3] = exp(lt * (2.0 / 3.0));
    v[F_GT + 5] = exp(-lt * (4.0 / 3.0));
    v[F_TRK] = -1.0 / t;
    v[F_AT + 0] = v[F_AT + 3] = -exp(-lt / 3.0) / 3.0;
    v[F_AT + 5] = 2.0 * exp(-lt * (7.0 / 3.0)) / 3.0;
  }
  const long long id = lin(g, i, j, k);
  for (int f = 0; f < NF; f++) y[f * g.fstride + id] = v[f];
}

cudaError_t launch_initial_data(const Grid& g, int kind, const double* p, int np, double* y,
                                cudaStream_t s) {
  IdParams ip{};
  ip.np = np < 33 ? np : 33;
  for (int q = 0; q < ip.np; q++) ip.p[q] = p[q];
  const long long total = (long long)g.sx * g.sy * g.sz;
  const int bs = 256;
  initial_data_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(g, kind, ip, y);
  return cudaGetLastError();
}

}  // namespace bssn
