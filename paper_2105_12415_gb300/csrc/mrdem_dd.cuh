// mrdem_dd.cuh -- double-float ("double-word") arithmetic on the FP32 units.
//
// GB300 runs FP64 at about 1/61 of its FP32 rate, so the final values of the
// FP32 form (closest points and distances of the comparison-based test of
// Sec. 3) are computed on pairs of floats x = hi + lo, |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum (Dekker 1971)
// and the FMA-based exact product; addition, multiplication and the products
// with a float follow the double-word algorithms analysed by Joldes, Muller
// and Popescu ("Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017): AccurateDWPlusDW (relative
// error < 3u^2 + 13u^3), DWTimesDW3 (< 4u^2) and DWTimesFP3 (< 2u^2), with
// u = 2^-24.  Division refines a float quotient by two residual corrections
// computed in double-word arithmetic; the square root takes one Newton step
// from the float root.  Every float operation below is an explicitly
// rounded intrinsic, so the compiler neither contracts nor reassociates them.
// Magnitudes must stay inside the float range with room for the low words
// (|x| in about [1e-30, 1e30]); callers scale their coordinates by a power of
// two to keep them there.
#pragma once

#include "mrdem_geometry.cuh"

namespace mrdem {

// The type is plain data (host code sizes arrays of it); the arithmetic below
// is device code.
struct dd {
  float hi, lo;
  dd() = default;
  MRDEM_HD constexpr dd(float h, float l) : hi(h), lo(l) {}
  MRDEM_HD dd(float h) : hi(h), lo(0.f) {}
  MRDEM_HD dd(int k) : hi((float)k), lo(0.f) {}
  MRDEM_HD dd(bool b) : hi(b ? 1.f : 0.f), lo(0.f) {}
  // from a double: the nearest float, then the float nearest the remainder;
  // infinities and NaN keep a zero low word
  MRDEM_HD dd(double x) : hi((float)x), lo(0.f) {
    if (isfinite(hi)) lo = (float)(x - (double)hi);
  }
};

#ifdef __CUDACC__
__device__ __forceinline__ double to_double(dd x) { return (double)x.hi + (double)x.lo; }

// Error-free transformations.
__device__ __forceinline__ dd two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd(s, e);
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return dd(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dd two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return dd(p, __fmaf_rn(a, b, -p));
}

// AccurateDWPlusDW.
__device__ __forceinline__ dd operator+(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  float c = __fadd_rn(s.lo, t.hi);
  dd v = fast_two_sum(s.hi, c);
  float w = __fadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ dd operator-(dd x) { return dd(-x.hi, -x.lo); }
__device__ __forceinline__ dd operator-(dd x, dd y) { return x + (-y); }
// DWTimesDW3.
__device__ __forceinline__ dd operator*(dd x, dd y) {
  dd c = two_prod(x.hi, y.hi);
  float tl0 = __fmul_rn(x.lo, y.lo);
  float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  float cl3 = __fadd_rn(c.lo, cl2);
  return fast_two_sum(c.hi, cl3);
}
// DWTimesFP3.
__device__ __forceinline__ dd mul_f(dd x, float y) {
  dd c = two_prod(x.hi, y);
  float cl3 = __fmaf_rn(x.lo, y, c.lo);
  return fast_two_sum(c.hi, cl3);
}
__device__ __forceinline__ dd operator*(int k, dd x) { return mul_f(x, (float)k); }
__device__ __forceinline__ dd operator*(bool b, dd x) { return b ? x : dd(0.f, 0.f); }

// x / y: float quotient q1 from a float reciprocal of y, then the residuals
// x - q1 y and (x - q1 y) - q2 y in double-word arithmetic give q2 and q3;
// each correction gains about 23 bits.
__device__ __forceinline__ dd operator/(dd x, dd y) {
  float r = __frcp_rn(y.hi);
  float q1 = __fmul_rn(x.hi, r);
  dd res = x - mul_f(y, q1);
  float q2 = __fmul_rn(res.hi, r);
  res = res - mul_f(y, q2);
  float q3 = __fmul_rn(res.hi, r);
  dd q = fast_two_sum(q1, q2);
  return q + dd(q3, 0.f);
}

// Comparisons of normalised values (hi = fl(hi + lo)): lexicographic.
__device__ __forceinline__ bool operator<(dd a, dd b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool operator>(dd a, dd b) { return b < a; }
__device__ __forceinline__ bool operator<=(dd a, dd b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(dd a, dd b) { return !(a < b); }
__device__ __forceinline__ bool operator==(dd a, dd b) { return a.hi == b.hi && a.lo == b.lo; }

// Square root: s = sqrt(hi) in float, one Newton correction
// (x - s^2) / (2 s) added in double-word arithmetic.
__device__ __forceinline__ dd dd_sqrt(dd x) {
  if (!(x.hi > 0.f)) return dd(0.f, 0.f);
  float s = __fsqrt_rn(x.hi);
  dd e = x - two_prod(s, s);
  float c = __fdiv_rn(e.hi, __fmul_rn(2.f, s));
  return fast_two_sum(s, c);
}

// Hooks of the geometry templates.
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ dd qdiv<dd>(dd a, dd b) { return a / b; }
template <>
__device__ __forceinline__ dd my_sqrt<dd>(dd v) { return dd_sqrt(v); }
#endif

__device__ __forceinline__ V3<dd> to_dd(V3<double> v) { return {dd(v.x), dd(v.y), dd(v.z)}; }
__device__ __forceinline__ V3<double> to_double(V3<dd> v) {
  return {to_double(v.x), to_double(v.y), to_double(v.z)};
}
#endif  // __CUDACC__

}  // namespace mrdem
