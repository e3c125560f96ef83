// mrdem_split.cuh -- a double as a double-float by integer operations.
//
// The contact kernels take FP64 inputs (closest points, positions, the
// force coefficients) and do their arithmetic in double-float on the FP32
// units.  Rounding a double to a float pair with floating-point conversions
// costs three operations on the FP64 pipe per value, about as much as the
// arithmetic it replaces, so split_double reads the IEEE 754 binary64
// encoding instead (sign, 11-bit biased exponent, 52-bit fraction) and
// builds the two floats with integer operations:
//   hi = the leading 24 significant bits of x (truncated),
//   lo = the next 24 significant bits (truncated),
// then renormalises the pair (|lo| <= ulp(hi)/2) with one Fast2Sum.  The
// pair holds x to better than 2^-47 |x|.  Zero and subnormal doubles give
// (0, 0); |x| beyond the float range gives (+-inf, 0), NaN a float NaN;
// a low word below the smallest normal float (|x| under about 2^-75) is
// dropped, leaving 2^-24 |x|.
#pragma once

#include <cstdint>
#include <cstring>

#include "mrdem_dd.cuh"

namespace mrdem {

MRDEM_HD float split_bits_to_float(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
#endif
}

MRDEM_HD int split_top_bit(uint32_t r) {  // r > 0
#ifdef __CUDA_ARCH__
  return 31 - __clz(r);
#else
  return 31 - __builtin_clz(r);
#endif
}

MRDEM_HD dd split_double(double x) {
  uint64_t b;
#ifdef __CUDA_ARCH__
  b = (uint64_t)__double_as_longlong(x);
#else
  std::memcpy(&b, &x, sizeof b);
#endif
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  const uint64_t f = b & 0xfffffffffffffull;
  if (e == 0) return dd(0.f, 0.f);
  if (e == 0x7ff) return dd(split_bits_to_float(sign | 0x7f800000u | (f ? 0x400000u : 0u)), 0.f);
  const int E = e - 1023 + 127;  // float exponent field of hi
  if (E >= 255) return dd(split_bits_to_float(sign | 0x7f800000u), 0.f);
  if (E <= 0) return dd(0.f, 0.f);
  float hi = split_bits_to_float(sign | ((uint32_t)E << 23) | (uint32_t)(f >> 29));
  const uint32_t r = (uint32_t)(f & 0x1fffffffu);  // the 29 fraction bits below hi's
  float lo = 0.f;
  if (r != 0) {
    // r units are 2^(e - 1023 - 52); its leading bit p sets lo's exponent
    const int p = split_top_bit(r);
    const int El = p + e - 1075 + 127;
    if (El > 0) {
      const uint32_t m = p >= 23 ? r >> (p - 23) : r << (23 - p);
      lo = split_bits_to_float(sign | ((uint32_t)El << 23) | (m & 0x7fffffu));
    }
  }
  // renormalise: Fast2Sum (|hi| >= |lo|)
#ifdef __CUDA_ARCH__
  const float s = __fadd_rn(hi, lo);
  return dd(s, __fsub_rn(lo, __fsub_rn(s, hi)));
#else
  const float s = hi + lo;
  return dd(s, lo - (s - hi));
#endif
}

MRDEM_HD V3<dd> split_double(V3<double> v) {
  return {split_double(v.x), split_double(v.y), split_double(v.z)};
}

}  // namespace mrdem
