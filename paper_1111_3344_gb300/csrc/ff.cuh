// Double-word ("float-float") arithmetic on the float32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// 48 significant bits.  On GB300 the float64 pipe issues some 58x fewer
// multiply-adds than the float32 pipe (1.25 against 73 TFLOP/s measured), so
// a right-hand side carried in double-word arithmetic costs fewer cycles
// than the same right-hand side in float64 while keeping its rounding error
// near 2^-47 of the operands -- close to float64's 2^-53, far from float's
// 2^-24.
//
// The building blocks are the published error-free transforms and
// double-word algorithms:
//  - TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2, Theorem B): s + e = a + b
//    exactly, six operations, no condition on the operands;
//  - FastTwoSum (Dekker 1971, "A floating-point technique for extending the
//    available precision"): the same in three operations when |a| >= |b|
//    (or a = 0);
//  - the exact product with a fused multiply-add: p = ab, e = fma(a, b, -p);
//  - double-word sum, product and quotient after Dekker (add2, mul2, div2)
//    in the forms analysed by Joldes, Muller and Popescu 2017 ("Tight and
//    rigorous error bounds for basic building blocks of double-word
//    arithmetic", ACM TOMS 44(2)).  The sum is Dekker's ("sloppy") form: its
//    error is at most a few 2^-48 of |x| + |y| (not of the result), which is
//    the error model of an ordinary float64 sum with 2^-53 replaced by about
//    2^-46.
// Every operation goes through the __f*_rn intrinsics, which the compiler
// never contracts into multiply-adds (a contraction would break the
// transforms).
#pragma once
#include <cuda_runtime.h>

namespace bssn {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // exact for small integers and every float; a double constant splits into
  // its leading float and the float nearest the remainder (folded at compile
  // time when the double is a literal)
  // (explicit: no silent conversion picks an ff overload for a double)
  __host__ __device__ explicit ff(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ explicit ff(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ explicit ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit ff(float2 v) : hi(v.x), lo(v.y) {}
  __host__ __device__ float2 f2() const { return make_float2(hi, lo); }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ ff ff_neg(ff x) { return ff(-x.hi, -x.lo); }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

// x * y: the exact product of the leading parts plus the cross terms
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// a * b + c with one renormalisation: the product's exact leading part and its
// error, summed into c by TwoSum
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, e;
  two_sum(p, c.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// x / y (Dekker's div2): the float quotient of the leading parts, then the
// quotient of the remainder x - q1 y (q1 y formed exactly) as a correction
__device__ __forceinline__ ff ff_div(ff x, ff y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const float p = __fmul_rn(y.hi, q1);
  const float pe = __fmaf_rn(y.hi, q1, -p);          // y.hi q1 = p + pe exactly
  // r = x - q1 y = (x.hi - p) - pe + x.lo - q1 y.lo; x.hi - p is exact (Sterbenz)
  float r = __fsub_rn(x.hi, p);
  r = __fsub_rn(r, pe);
  r = __fadd_rn(r, x.lo);
  r = __fmaf_rn(-q1, y.lo, r);
  const float q2 = __fdiv_rn(r, y.hi);
  ff o;
  fast_two_sum(q1, q2, o.hi, o.lo);
  return o;
}

__device__ __forceinline__ ff operator+(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return ff_sub(a, b); }
__device__ __forceinline__ ff operator*(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ ff operator/(ff a, ff b) { return ff_div(a, b); }
__device__ __forceinline__ ff operator-(ff a) { return ff_neg(a); }
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = ff_add(a, b); }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = ff_sub(a, b); }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = ff_mul(a, b); }
// comparisons: hi carries the sign and, unless the two his are equal, the order
__device__ __forceinline__ bool operator>(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(ff a, ff b) { return b > a; }
__device__ __forceinline__ bool operator>=(ff a, ff b) { return !(b > a); }
__device__ __forceinline__ bool operator<=(ff a, ff b) { return !(a > b); }
__device__ __forceinline__ ff ff_fabs(ff a) { return a.hi < 0.0f ? ff_neg(a) : a; }

// conversions to and from float64 (float64-pipe instructions: used once per
// value at the combine, never inside the right-hand side)
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_from_double(double d) {
  const float h = __double2float_rn(d);
  return ff(h, __double2float_rn(d - (double)h));
}
// exp through float64 (the phi variant only, once per point)
__device__ __forceinline__ ff ff_exp(ff a) { return ff_from_double(::exp(ff_to_double(a))); }

}  // namespace bssn
