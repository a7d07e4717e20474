// FP32 <-> FP64 conversions on the integer pipe (the mixed form's FP64
// accumulator), shared by the kernels and by the conversion check.
#pragma once

#include <cstdint>

namespace frgb {

// Conversions between binary32 and binary64 on the integer pipe, written
// from the IEEE 754 layouts (sign | biased exponent | fraction; biases 127
// and 1023, fractions of 23 and 52 bits).  Only the FP64 accumulator of the
// mixed form needs them: GB300 issues FP64 instructions, conversions to and
// from FP64 included, at a small fraction of its FP32 rate.  Inputs outside
// the fast path's range take the hardware conversion, so both are exact
// (widening) and round to nearest even (narrowing) for every input.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double(int(b), 0);  // +-0
  if (e - 1u >= 254u) return double(f);  // subnormal, infinite, NaN
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xfffffu);
  return __hiloint2double(int(hi), int(b << 29));
}

__device__ __forceinline__ float narrow_f64(double d) {
  const uint32_t hi = uint32_t(__double2hiint(d)), lo = uint32_t(__double2loint(d));
  const uint32_t e = (hi >> 20) & 0x7ffu;
  // the result's exponent e - 896 must be a normal one, 1..254
  if (e - 897u >= 254u) return __double2float_rn(d);
  uint32_t body = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu;  // the 29 fraction bits dropped
  body += uint32_t(rem > 0x10000000u) | (uint32_t(rem == 0x10000000u) & body);
  return __uint_as_float((hi & 0x80000000u) | body);
}

// 1/x for positive normal x by Newton-Raphson from the FP32 reciprocal of
// xf = x rounded to FP32: r <- r + r (1 - x r), twice, each step squaring
// the relative error (2^-23 -> 2^-46 -> below FP64 rounding), four FP64
// FMAs instead of the FP64 division's longer sequence.  Within 2 units in
// the last place of the correctly rounded 1/x (checked on the GPU against
// the division by fr_check_conversions).  x outside [2^-125, 2^126) takes
// the division.
__device__ __forceinline__ double rcp64(double x, float xf) {
  const int ex = int((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
  if (ex < -125 || ex > 125) return 1.0 / x;
  double r = widen_f32(__frcp_rn(xf));
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// y^(1/5), the sign of y kept, for normal y: with |y| = m 2^(5k), m in
// [1, 32), the root is m^(1/5) 2^k; m^(1/5) comes from the FP32 fifth root
// (relative error ~1e-7) and two Newton steps on x^5 = m,
// x <- x - (x^5 - m) / (5 x^4), each roughly squaring the error.  A few
// FP64 operations instead of an FP64 pow; r^5 = |y| to 5e-15 relative
// (checked on the GPU by fr_check_conversions).  Zero, subnormal, infinite
// and NaN y take the pow.
__device__ __forceinline__ double root5(double y) {
  const long long b = __double_as_longlong(y) & 0x7fffffffffffffffLL;
  const int e = int(b >> 52) - 1023;
  if (e <= -1023 || e >= 1024) return y < 0.0 ? -pow(-y, 0.2) : pow(y, 0.2);
  const int k = e >= 0 ? e / 5 : -((4 - e) / 5);  // floor(e / 5)
  const double m = __longlong_as_double(b - ((long long)(5 * k) << 52));
  double x = widen_f32(powf(narrow_f64(m), 0.2f));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double x2 = x * x, x4 = x2 * x2, d = 5.0 * x4;
    x = fma(-fma(x4, x, -m), rcp64(d, narrow_f64(d)), x);
  }
  const double r = __longlong_as_double(__double_as_longlong(x) + ((long long)k << 52));
  return y < 0.0 ? -r : r;
}

}  // namespace frgb
