/*
 * bssn_oracle_instrumented.cpp -- the oracle's point-wise right-hand side
 * (bssn_rhs.h, Sec. "Spacetime Curvature Evolution" and Sec. "Boundary
 * Conditions") evaluated with an instrumented arithmetic type.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the CUDA library never
 * calls, links or includes it.
 *
 * The type `real` below carries three things through the same expressions,
 * in the same order, as the plain float64 oracle:
 *  - v: the float64 value, by the same IEEE operations (build with
 *    -ffp-contract=off), so it equals the plain oracle's result bit for bit;
 *  - m: the magnitude of the expression evaluated on absolute values --
 *    every leaf (state value or constant) replaced by |leaf|, every
 *    difference by a sum.  For +, - and * this is the quantity that bounds
 *    the rounding error of any evaluation order of the same sum of products:
 *    |fl(e) - e| <= gamma_n m with gamma_n = n u / (1 - n u), u = 2^-53, n the
 *    depth of the expression (Higham, "Accuracy and Stability of Numerical
 *    Algorithms", 2nd ed., Sec. 3.1-3.3).  A quotient a / b propagates the
 *    relative errors of both operands: m = (m_a + |a/b| m_b) / |b|; a square
 *    root m = |sqrt a| + m_a / (2 |sqrt a|); an exponential
 *    m = |exp a| (1 + m_a).
 *  - operation counts (add/subtract, multiply, divide, sqrt/exp) of the
 *    printed arrangement, per thread.
 * The same header is also compiled with long double arithmetic (namespace
 * ext), so that the float64 evaluation can be compared with one of a much
 * smaller unit roundoff.
 */
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>

namespace {

thread_local long long n_add = 0, n_mul = 0, n_div = 0, n_fun = 0;

struct real {
  double v;  // value
  double m;  // magnitude of the absolute-value evaluation
  real() : v(0.0), m(0.0) {}
  real(double x) : v(x), m(std::fabs(x)) {}  // a leaf: state value or constant
  static real make(double v, double m) {
    real r;
    r.v = v;
    r.m = m;
    return r;
  }
};

inline real operator+(real a, real b) { n_add++; return real::make(a.v + b.v, a.m + b.m); }
inline real operator-(real a, real b) { n_add++; return real::make(a.v - b.v, a.m + b.m); }
inline real operator*(real a, real b) { n_mul++; return real::make(a.v * b.v, a.m * b.m); }
inline real operator/(real a, real b) {
  n_div++;
  const double q = a.v / b.v;
  return real::make(q, (a.m + std::fabs(q) * b.m) / std::fabs(b.v));
}
inline real operator-(real a) { return real::make(-a.v, a.m); }
inline real operator+(real a, double b) { return a + real(b); }
inline real operator-(real a, double b) { return a - real(b); }
inline real operator*(real a, double b) { return a * real(b); }
inline real operator/(real a, double b) { return a / real(b); }
inline real operator+(double a, real b) { return real(a) + b; }
inline real operator-(double a, real b) { return real(a) - b; }
inline real operator*(double a, real b) { return real(a) * b; }
inline real operator/(double a, real b) { return real(a) / b; }
inline real& operator+=(real& a, real b) { return a = a + b; }
inline real& operator-=(real& a, real b) { return a = a - b; }
inline real& operator*=(real& a, real b) { return a = a * b; }
inline real& operator/=(real& a, real b) { return a = a / b; }
inline bool operator>(real a, double b) { return a.v > b; }
inline bool operator>=(real a, double b) { return a.v >= b; }
inline bool operator<(real a, double b) { return a.v < b; }
inline bool operator<=(real a, double b) { return a.v <= b; }
inline real sqrt(real a) {
  n_fun++;
  const double s = std::sqrt(a.v);
  return real::make(s, s + (s > 0.0 ? a.m / (2.0 * s) : 0.0));
}
inline real exp(real a) {
  n_fun++;
  const double e = std::exp(a.v);
  return real::make(e, e * (1.0 + a.m));
}
inline real fabs(real a) { return real::make(std::fabs(a.v), a.m); }
using std::exp;
using std::fabs;
using std::sqrt;
using std::isinf;

#include "bssn_rhs.h"

}  // namespace

// The same header once more in long double (x87 extended on x86-64, IEEE
// quad on aarch64): an evaluation with a far smaller unit roundoff, against
// which the float64 evaluation's rounding error is measured.
#undef BSSN_ORACLE_RHS_H
namespace ext {
typedef long double real;
using std::exp;
using std::fabs;
using std::isinf;
using std::sqrt;
#include "bssn_rhs.h"
}  // namespace ext

extern "C" {

/* Right-hand side at stored points ijk[3p + d] (as oracle_rhs_points), with
 * val[p NF + f] the float64 value and mag[p NF + f] the magnitude of its
 * absolute-value evaluation. */
void oracle_rhs_points_mag(const ocfg* c, const double* st, int np, const int* ijk, double* val,
                           double* mag) {
#pragma omp parallel for schedule(dynamic)
  for (int p = 0; p < np; p++) {
    real out[NF];
    rhs_at(c, st, ijk[3 * p], ijk[3 * p + 1], ijk[3 * p + 2], out);
    for (int f = 0; f < NF; f++) {
      val[(size_t)p * NF + f] = out[f].v;
      mag[(size_t)p * NF + f] = out[f].m;
    }
  }
}

/* Right-hand side at stored points ijk in long double, rounded to double at
 * the end: out[p NF + f]. */
void oracle_rhs_points_ext(const ocfg* c, const double* st, int np, const int* ijk, double* out) {
  const ext::ocfg* ce = reinterpret_cast<const ext::ocfg*>(c);
#pragma omp parallel for schedule(dynamic)
  for (int p = 0; p < np; p++) {
    long double o[NF];
    ext::rhs_at(ce, st, ijk[3 * p], ijk[3 * p + 1], ijk[3 * p + 2], o);
    for (int f = 0; f < NF; f++) out[(size_t)p * NF + f] = (double)o[f];
  }
}

/* Operations of one right-hand-side evaluation at stored point (i, j, k), in
 * the printed arrangement: counts[0] additions and subtractions, [1]
 * multiplications, [2] divisions, [3] square roots and exponentials. */
void oracle_rhs_opcount(const ocfg* c, const double* st, int i, int j, int k, long long counts[4]) {
  n_add = n_mul = n_div = n_fun = 0;
  real out[NF];
  rhs_at(c, st, i, j, k, out);
  counts[0] = n_add;
  counts[1] = n_mul;
  counts[2] = n_div;
  counts[3] = n_fun;
}

}  // extern "C"
