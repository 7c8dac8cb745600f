// Double-double ("double-word") arithmetic on the binary64 units: a value is
// the unevaluated sum hi + lo of two binary64 numbers with |lo| <= ulp(hi)/2,
// about 106 significant bits. The building blocks are the error-free
// transformations TwoSum (Knuth), FastTwoSum (Dekker) and TwoProd by a fused
// multiply-add; the sum and product of two double-words follow the
// algorithms of Joldes, Muller and Popescu, "Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic", ACM TOMS 44 (2017):
// the accurate sum (their Algorithm 6, relative error <= 3u^2) and the
// product with FMA (Algorithm 12, <= 4u^2), u = 2^-53. Division is long
// division with two correction steps and the square root one Newton step
// from the binary64 root (Karp and Markstein, ACM TOMS 23, 1997).
//
// Every operation is written with the _rn intrinsics so that the compiler
// neither contracts nor reorders the steps the transformations rely on.
#pragma once
#include <cuda_runtime.h>

namespace mpsgb {

struct __align__(16) dd {
  double hi, lo;
};
struct __align__(16) cdd {
  dd re, im;
};

// binary64 operations counted per double-word operation (for the executed
// flop count of the kernels that use them)
constexpr int kFlopsDdAdd = 20;
constexpr int kFlopsDdMul = 9;
constexpr int kFlopsCddMul = 4 * kFlopsDdMul + 2 * kFlopsDdAdd;

__device__ __forceinline__ dd dd_make(double a) { return dd{a, 0.0}; }

__device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return dd{s, e};
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  return dd{s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
  const double p = __dmul_rn(a, b);
  return dd{p, __fma_rn(a, b, -p)};
}

__device__ __forceinline__ dd dd_add(dd x, dd y) {
  const dd s = two_sum(x.hi, y.hi);
  const dd t = two_sum(x.lo, y.lo);
  const dd v = fast_two_sum(s.hi, __dadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __dadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

__device__ __forceinline__ dd dd_add_d(dd x, double y) {
  const dd s = two_sum(x.hi, y);
  const dd v = fast_two_sum(s.hi, __dadd_rn(x.lo, s.lo));
  return v;
}

__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const dd c = two_prod(x.hi, y.hi);
  const double t1 = __fma_rn(x.hi, y.lo, __dmul_rn(x.lo, y.lo));
  const double t2 = __fma_rn(x.lo, y.hi, t1);
  return fast_two_sum(c.hi, __dadd_rn(c.lo, t2));
}

__device__ __forceinline__ dd dd_mul_d(dd x, double y) {
  const dd c = two_prod(x.hi, y);
  return fast_two_sum(c.hi, __fma_rn(x.lo, y, c.lo));
}

__device__ __forceinline__ dd dd_sqr(dd x) {
  const dd c = two_prod(x.hi, x.hi);
  const double t = __dmul_rn(__dadd_rn(x.hi, x.hi), x.lo);
  return fast_two_sum(c.hi, __dadd_rn(c.lo, t));
}

__device__ __forceinline__ dd dd_div(dd x, dd y) {
  const double q1 = __ddiv_rn(x.hi, y.hi);
  dd r = dd_sub(x, dd_mul_d(y, q1));
  const double q2 = __ddiv_rn(r.hi, y.hi);
  r = dd_sub(r, dd_mul_d(y, q2));
  const double q3 = __ddiv_rn(r.hi, y.hi);
  return dd_add_d(fast_two_sum(q1, q2), q3);
}

__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (!(a.hi > 0.0)) return dd{0.0, 0.0};
  const double s = __dsqrt_rn(a.hi);
  const dd r = dd_sub(a, two_prod(s, s));
  return fast_two_sum(s, __ddiv_rn(r.hi, __dadd_rn(s, s)));
}

__device__ __forceinline__ bool dd_gt(dd a, dd b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

__device__ __forceinline__ cdd cdd_make(double re, double im) { return cdd{dd{re, 0.0}, dd{im, 0.0}}; }
__device__ __forceinline__ cdd cdd_add(cdd x, cdd y) { return cdd{dd_add(x.re, y.re), dd_add(x.im, y.im)}; }
__device__ __forceinline__ cdd cdd_sub(cdd x, cdd y) { return cdd{dd_sub(x.re, y.re), dd_sub(x.im, y.im)}; }
__device__ __forceinline__ cdd cdd_conj(cdd x) { return cdd{x.re, dd_neg(x.im)}; }
__device__ __forceinline__ cdd cdd_mul(cdd x, cdd y) {
  return cdd{dd_sub(dd_mul(x.re, y.re), dd_mul(x.im, y.im)), dd_add(dd_mul(x.re, y.im), dd_mul(x.im, y.re))};
}
// conj(x) * y
__device__ __forceinline__ cdd cdd_cmul(cdd x, cdd y) {
  return cdd{dd_add(dd_mul(x.re, y.re), dd_mul(x.im, y.im)), dd_sub(dd_mul(x.re, y.im), dd_mul(x.im, y.re))};
}
__device__ __forceinline__ cdd cdd_scale(dd s, cdd x) { return cdd{dd_mul(s, x.re), dd_mul(s, x.im)}; }
__device__ __forceinline__ dd cdd_abs2(cdd x) { return dd_add(dd_sqr(x.re), dd_sqr(x.im)); }

__device__ __forceinline__ dd shfl_xor_dd(dd v, int m) {
  return dd{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

}  // namespace mpsgb
