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

}  // namespace frgb
