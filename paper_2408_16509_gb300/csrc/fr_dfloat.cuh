// Double-float arithmetic (a value carried as an unevaluated sum hi + lo of
// two FP32 numbers, |lo| <= ulp(hi) / 2): Dekker's exact product via a
// fused multiply-add and Knuth's exact two-sum (Dekker 1971, "A
// floating-point technique for extending the available precision";
// Knuth, TAOCP vol. 2, 4.2.2).  About 46 significant bits on the FP32
// pipe, which GB300 issues some 60x faster than its FP64 pipe.
//
// The entropy filter uses it to find, among the points of an element, the
// one of least pressure or least entropy (the ordering key below); the
// value at that point is then computed in FP64.
#pragma once
#include <cstdint>

#include "fr_convert.cuh"

namespace frgb {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_two_prod(float a, float b) {
  const float p = a * b;
  return dfl{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfl{s, (a - (s - bb)) + (b - bb)};
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfl{s, b - (s - a)};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const dfl s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const dfl p = df_two_prod(x.hi, y.hi);
  return df_fast_two_sum(p.hi, p.lo + (x.hi * y.lo + x.lo * y.hi));
}

// 1/a for a normal positive float: the FP32 quotient and its residual
// 1 - a r (exact through the fused multiply-add)
__device__ __forceinline__ dfl df_rcp(float a) {
  const float r = 1.0f / a;
  const float e = fmaf(-a, r, 1.0f);
  return df_fast_two_sum(r, r * e);
}

// the double-float's value as an FP64 number (one FP64 add)
__device__ __forceinline__ double df_to_f64(dfl x) { return widen_f32(x.hi) + widen_f32(x.lo); }

// p = (gamma - 1)(E - (mx^2 + my^2 + mz^2) / (2 rho)) from FP32 conserved
// values (exact inputs) with rho > 0 and rr = 1/rho; gm1 = gamma - 1 as a
// double-float.  *amb: |p| is within 2^-36 of (|E| + |k|), where the
// cancellation leaves too few bits to order or sign p; the caller then
// takes the FP64 formula.
__device__ __forceinline__ dfl df_pressure(float mx, float my, float mz, float E, dfl rr,
                                           dfl gm1, bool* amb) {
  const dfl m2 = df_add(df_add(df_two_prod(mx, mx), df_two_prod(my, my)), df_two_prod(mz, mz));
  const dfl k = df_mul(dfl{0.5f * m2.hi, 0.5f * m2.lo}, rr);
  const dfl q = df_add(dfl{E, 0.f}, dfl{-k.hi, -k.lo});
  *amb = !(fabsf(q.hi) > 0x1p-36f * (fabsf(E) + fabsf(k.hi)));
  return df_mul(gm1, q);
}

// Scale x = m 2^e with m in [1, 2) (x normal and nonzero, taken as |x|);
// returns m as a double-float and e.
__device__ __forceinline__ dfl df_normalise(dfl x, int* e) {
  const float a = fabsf(x.hi);
  const int ex = int((__float_as_uint(a) >> 23) & 0xffu) - 127;
  const float s = __uint_as_float(uint32_t(127 - ex) << 23);  // 2^-ex, exact
  *e = ex;
  const float sg = x.hi < 0.f ? -1.f : 1.f;
  return dfl{a * s, sg * x.lo * s};
}

// Ordering key of s^5 = p^5 rho^-7 (gamma = 7/5) as an FP64 number, from
// double-float p and rr = 1/rho: sign(p) |p|^5 rr^7 to about 2^-43
// relative.  Returns false (no key) when an exponent leaves the ranges
// where every intermediate stays a normal FP32 / FP64 number.
__device__ __forceinline__ bool df_s5_key(dfl p, dfl rr, double* key) {
  const int ep0 = int((__float_as_uint(fabsf(p.hi)) >> 23) & 0xffu);
  const int er0 = int((__float_as_uint(rr.hi) >> 23) & 0xffu);
  if (ep0 < 30 || ep0 > 225 || er0 < 30 || er0 > 225) return false;
  int ep, er;
  const dfl P = df_normalise(p, &ep), R = df_normalise(rr, &er);
  const dfl P2 = df_mul(P, P), P4 = df_mul(P2, P2), P5 = df_mul(P4, P);
  const dfl R2 = df_mul(R, R), R4 = df_mul(R2, R2), R7 = df_mul(df_mul(R4, R2), R);
  const int E = 5 * ep + 7 * er;
  if (E < -1000 || E > 1000) return false;  // m 2^E normal in FP64
  const dfl M = df_mul(P5, R7);  // in [1, 2^12)
  const double m = df_to_f64(M);
  const long long b = __double_as_longlong(m) + ((long long)E << 52);
  const double y = __longlong_as_double(b);
  *key = p.hi < 0.f ? -y : y;
  return true;
}

}  // namespace frgb
