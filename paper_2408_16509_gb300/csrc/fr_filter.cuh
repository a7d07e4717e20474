// Entropy filter with a learned start guess (PyFR v2.0.3, Section 3.2).
//
// The paper filters, per element, the high modes of the solution when it
// violates positivity of density or pressure or a minimum-entropy
// condition, with the filter strength found iteratively so that as little
// filtering as possible is applied.  Reading used here (no formulas in the
// paper):
//   u^ = V^{-1} u in the orthonormal modal basis, u^_k <- exp(-zeta
//   (d_k/p)^2) u^_k with d_k the total degree (the mean is untouched);
//   constraints at solution and flux points: rho >= 1e-8, p >= 1e-8,
//   s = p rho^-gamma >= s_min - 1e-8 s_min, s_min = min of s over the stage
//   input at the element's solution points, own flux points and the partner
//   flux points across its faces;
//   margin g(zeta) = min((rho-1e-8)/rho_mean, (p-1e-8)/p_mean,
//   (s - s_min + 1e-8 s_min)/s_min), evaluated in FP64;
//   zeta* = the smallest feasible strength, by a bracketed Illinois
//   iteration (ended when the feasible end's margin is at most the entropy
//   tolerance below, or at relative width 1e-6, or after 24 evaluations)
//   started from [0, 36] or from a predicted guess z0 (bracket opened at
//   z0, then z0 / r or r z0 with r = 1.25 by default, then halving /
//   doubling).
//   The entropy tolerance is 1e-8 for FP64 stage values and 2^-20 for FP32
//   ones (1e-8 is below FP32 resolution, where the decision would be made
//   by rounding noise).
// The predictor: 4 element features -> Linear(4,32)-SiLU-Linear(32,32)-SiLU
// -Linear(32,1)-softplus, BF16 weights and FP32 accumulation.
#pragma once
#include <cuda_bf16.h>

#include <type_traits>

#include "fr_dfloat.cuh"
#include "fr_kernels.cuh"

namespace frgb {

constexpr int kMlpH = 32;
constexpr int kMlpIn = 4;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH +
                           kMlpH + 1 + 2 * kMlpIn;  // 1257
constexpr int kMlpTrain = kMlpParams - 2 * kMlpIn;   // 1249
// offsets in the parameter vector
constexpr int kW1 = 0, kB1 = kW1 + kMlpH * kMlpIn, kW2 = kB1 + kMlpH,
              kB2 = kW2 + kMlpH * kMlpH, kW3 = kB2 + kMlpH, kB3 = kW3 + kMlpH,
              kMean = kB3 + 1, kStd = kMean + kMlpIn;

constexpr double kZetaMax = 36.0;
constexpr double kEpsPos = 1e-8;
constexpr double kRelTol = 1e-6;
constexpr int kMaxEvals = 24;
// threads of a k_filter CTA: one point per thread for p = 3 hexahedra (64
// solution + 96 flux points), two for p = 4
constexpr int kFilterThreads = 160;

struct FilterStats {
  unsigned long long filtered;    // element-stages filtered (zeta > 0)
  unsigned long long evals;       // margin evaluations in those
  unsigned long long fallbacks;   // elements filtered with zeta_max
  unsigned long long samples;     // training samples written
  unsigned long long guessed;     // element-stages that used the predictor
};

template <typename T>
struct FilterOps {
  const T* VinvT;   // [nu][nm]   modal <- nodal, transposed
  const T* VT;      // [nm][nu+nf] nodal (solution then flux points) <- modal
  const T* deg;     // [nm] mode degree / p
  const T* W;       // [nu] integration weights
  const int32_t* partner;  // [ne][nf] partner flux-point code or -1
};

struct FilterArgs {
  double gamma;
  double tau;            // relative entropy tolerance
  double ratio;          // first bracket step around a predicted guess
  float* zeta_last;      // [ne] zeta of the last filtered stage (0: none)
  int* evals_last;       // [ne] margin evaluations of the last stage
  double* smin;          // [ne] of this type
  FilterStats* stats;
  float* samples;        // [cap][5] (4 features, zeta*)
  unsigned long long cap;
  const __nv_bfloat16* mlp;  // predictor weights or nullptr
  const float* mlp_norm;     // mean[4], std[4]
};

// Entropy minima without an FP64 pow per point (gamma = 7/5, the value
// every workload here uses).  Then s^5 = p^5 rho^-7 exactly, and x -> x^5
// is increasing on all reals, so the point of least s is the point of
// least y = p^5 (1/rho)^7, formed with seven FP64 multiplications; s_min =
// y_min^(1/5) is one fifth root per minimum (root5: Newton steps from the
// FP32 root), and a sign test s >= b is y >= b^5.  Against p rho^-gamma
// evaluated per point this differs only by rounding (about 1e-15
// relative; FP64 1.4 itself is 7/5 to 6e-17).  y is formed only where it
// stays a normal FP64 number (s5_in_range); other points take the
// per-point pow.
__device__ __forceinline__ bool entropy_by_s5(double g) { return g == 1.4; }

// unbiased binary exponent of x from its bits (integer pipe)
__device__ __forceinline__ int dexp2(double x) {
  return int((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}

// |p| in [2^-99, 2^100) or p = 0, 1/rho in [2^-69, 2^70): then p^5 (1/rho)^7
// is a normal number (between 2^-978 and 2^985); tested on the exponent
// bits, off the FP64 pipe
__device__ __forceinline__ bool s5_in_range(double p, double rr) {
  const long long pb = __double_as_longlong(p) & 0x7fffffffffffffffLL;
  const int ep = dexp2(p), er = dexp2(rr);
  return (pb == 0 || (ep >= -99 && ep <= 99)) && er >= -69 && er <= 69;
}

// minimum of two doubles by their order-preserving integer keys (defined
// below for the block reductions), off the FP64 pipe
__device__ __forceinline__ long long dkey(double x);
__device__ __forceinline__ double dunkey(long long k);
__device__ __forceinline__ double dmin_key(double a, double b) {
  // like fmin: a NaN operand is ignored
  const long long mag = __double_as_longlong(b) & 0x7fffffffffffffffLL;
  if (mag > 0x7ff0000000000000LL) return a;
  return dunkey(min(dkey(a), dkey(b)));
}

// FP64 copy of a stored value: FP32 values are widened on the integer pipe
template <typename S>
__device__ __forceinline__ double to_f64(S x) {
  if constexpr (sizeof(S) == 4) return widen_f32(x);
  else return double(x);
}

__device__ __forceinline__ double s5_of(double p, double rr) {
  const double p2 = p * p, r2 = rr * rr, r4 = r2 * r2;
  return (p2 * p2 * p) * (r4 * r2 * rr);
}

__device__ __forceinline__ double s_of_s5(double y) {
  if (!(y == y) || y == INFINITY || y == -INFINITY) return y;
  return root5(y);
}

// FP32 screen of a point for the exact FP64 minima of p and s = p rho^-g.
// From the state rounded to FP32, p32 and a bound dp with |p32 - p| <= dp
// (p the FP64 pressure of the same state): every operation of
// p = (g-1)(E - (mx^2+my^2+mz^2)/(2 rho)) and the rounding of the inputs
// contribute at most ~11 unit roundoffs (2^-24) of (g-1)(|E| + |k|); dp
// takes 2e-6 ~ 34 of them.  __powf(rho, -g) = 2^(-g log2 rho) errs by
// about ln 2 |g log2 rho| 2^-22 relative, under 2e-6 for rho in [2^-8, 2^8];
// the s bounds widen it to 1e-5 there.  Points with rho outside that range
// get no entropy bounds, points with rho <= 0 (or NaN) no bounds at all.
struct PtScreen {
  float plo, phi, slo, shi;
  bool pos;  // rho > 0 in FP32 (bounds valid)
};

__device__ __forceinline__ PtScreen screen_point(float r, float mx, float my,
                                                 float mz, float E, float g) {
  PtScreen o;
  o.pos = r > 0.f;
  if (!o.pos) {
    o.plo = o.slo = -INFINITY;
    o.phi = o.shi = INFINITY;
    return o;
  }
  const float k = 0.5f * (mx * mx + my * my + mz * mz) / r;
  const float gm1 = g - 1.f;
  const float p = gm1 * (E - k);
  const float dp = 2e-6f * gm1 * (fabsf(E) + fabsf(k));
  o.plo = p - dp;
  o.phi = p + dp;
  if (!(r >= 0x1p-8f && r <= 0x1p8f)) {
    // the intrinsic's error grows with |g log2 r|: outside this range the
    // 1e-5 margin is not shown to hold, so no entropy bounds (the point's
    // FP64 entropy is always evaluated)
    o.slo = -INFINITY;
    o.shi = INFINITY;
    return o;
  }
  const float rg = __powf(r, -g);
  o.slo = o.plo * rg * (o.plo >= 0.f ? 1.f - 1e-5f : 1.f + 1e-5f);
  o.shi = o.phi * rg * (o.phi >= 0.f ? 1.f + 1e-5f : 1.f - 1e-5f);
  return o;
}

__device__ __forceinline__ double pressure64(const double v[5], double g) {
  return (g - 1.0) * (v[4] - 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / v[0]);
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// s_min per element from the stage input: one warp per element, over the
// element's solution and flux points and its face neighbours' flux points,
// s = p rho^-g at the admissible points (rho > 0, p > 0), 0 when there are
// none.  Every point is screened in FP32 (screen_point); the FP64 value is
// computed only where the screen cannot exclude the minimum or cannot decide
// admissibility, so the result equals the all-FP64 minimum.
template <typename T, typename TR, int NU, int NF>
__global__ void k_entropy_min(long long ne, const T* __restrict__ uin,
                              const TR* __restrict__ X,
                              const T* __restrict__ uf_all, TypeTab tt,
                              int tidx, const int32_t* __restrict__ partner,
                              double gamma, double* __restrict__ smin) {
  constexpr int NQ = (NU + 2 * NF + 31) / 32;
  const int lane = threadIdx.x & 31;
  const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= ne) return;
  const T* uf = uf_all + tt.off_f[tidx];
  // state at point slot i, converted to V (float for the screen, double
  // for the exact value); false when the slot holds no point
  auto load = [&](int i, auto* v) -> bool {
    using V = std::remove_pointer_t<decltype(v)>;
    if (i < NU) {
#pragma unroll
      for (int k = 0; k < 5; ++k)
        v[k] = uin ? V(uin[(e * 5 + k) * NU + i]) : V(X[(e * 5 + k) * NU + i]);
      return true;
    }
    if (i < NU + NF) {
      const int f = i - NU;
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = V(uf[(e * 5 + k) * NF + f]);
      return true;
    }
    if (i < NU + 2 * NF) {
      const int32_t c = partner[e * NF + (i - NU - NF)];
      if (c < 0) return false;
      int t2, f2;
      long long e2;
      decode_fp(c, tt, &t2, &e2, &f2);
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = V(uf_all[fp_index(tt, t2, e2, f2, 5, k)]);
      return true;
    }
    return false;
  };
  const float gf = float(gamma);
  float slo[NQ];
  uint32_t cand = 0;  // bit q: slot q needs the FP64 value
  float shi_min = INFINITY;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    slo[q] = INFINITY;
    float v[5];
    if (!load(lane + 32 * q, v)) continue;
    const PtScreen sc = screen_point(v[0], v[1], v[2], v[3], v[4], gf);
    if (!sc.pos || sc.phi <= 0.f) {
      // p < 0 for sure: not admissible.  rho <= 0 in FP32: FP64 decides
      // (an FP64 density can round to zero in FP32)
      if (!sc.pos) cand |= 1u << q;
      continue;
    }
    if (sc.plo <= 0.f) {  // admissibility undecided
      cand |= 1u << q;
      continue;
    }
    slo[q] = sc.slo;
    shi_min = fminf(shi_min, sc.shi);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    shi_min = fminf(shi_min, __shfl_xor_sync(0xffffffffu, shi_min, o));
  const bool by5 = entropy_by_s5(gamma);
  // the stored values as FP64: FP32 stage values widened exactly on the
  // integer pipe (the FP64 pipe is this kernel's bound)
  constexpr bool f32in = sizeof(T) == 4 && sizeof(TR) == 4;
  if constexpr (f32in) {
    if (by5) {
      // FP32 values, gamma = 7/5: the point of least s^5 is selected in
      // double-float arithmetic (FP64 where the pressure is too close to
      // zero to sign), then s^5 is computed in FP64 at that point
      const float gm1h = float(gamma - 1.0);
      const dfl gm1d{gm1h, float((gamma - 1.0) - widen_f32(gm1h))};
      double m = INFINITY;  // direct minimum (points outside the s^5 range)
      long long ky = 0x7fffffffffffffffLL;
      int qy = -1;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if (!((cand >> q) & 1u) && !(slo[q] <= shi_min)) continue;
        float vf[5];
        if (!load(lane + 32 * q, vf)) continue;
        if (!(vf[0] > 0.f)) continue;
        bool amb = !(vf[0] >= 0x1p-100f && vf[0] <= 0x1p100f);
        dfl rr{0.f, 0.f}, pd{0.f, 0.f};
        if (!amb) {
          rr = df_rcp(vf[0]);
          pd = df_pressure(vf[1], vf[2], vf[3], vf[4], rr, gm1d, &amb);
        }
        double yk;
        bool ykey = false;
        if (amb) {
          double v[5];
#pragma unroll
          for (int k = 0; k < 5; ++k) v[k] = widen_f32(vf[k]);
          const double rr64 = rcp64(v[0], vf[0]);
          const double p = (gamma - 1.0) * (v[4] - 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) * rr64);
          if (!(p > 0.0)) continue;
          if (s5_in_range(p, rr64)) {
            yk = s5_of(p, rr64);
            ykey = true;
          } else {
            m = dmin_key(m, p * pow(v[0], -gamma));
          }
        } else {
          if (!(pd.hi > 0.f)) continue;
          if (df_s5_key(pd, rr, &yk)) {
            ykey = true;
          } else {
            double v[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) v[k] = widen_f32(vf[k]);
            m = dmin_key(m, pressure64(v, gamma) * pow(v[0], -gamma));
          }
        }
        if (ykey) {
          const long long kt = (dkey(yk) & ~0x1fLL) | lane;
          if (kt < ky) {
            ky = kt;
            qy = q;
          }
        }
      }
      long long km = dkey(m), kym = ky;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        km = min(km, __shfl_xor_sync(0xffffffffu, km, o));
        kym = min(kym, __shfl_xor_sync(0xffffffffu, kym, o));
      }
      m = dunkey(km);
      // the selected point's s^5 in FP64, on its lane, then to lane 0
      double ysel = INFINITY, sdir = INFINITY;
      if (qy >= 0 && ky == kym) {
        float vf[5];
        load(lane + 32 * qy, vf);
        double v[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = widen_f32(vf[k]);
        const double rr64 = rcp64(v[0], vf[0]);
        const double p = (gamma - 1.0) * (v[4] - 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) * rr64);
        if (s5_in_range(p, rr64)) ysel = s5_of(p, rr64);
        else sdir = p * pow(v[0], -gamma);
      }
      const int src = kym == 0x7fffffffffffffffLL ? 0 : int(kym & 0x1f);
      ysel = __shfl_sync(0xffffffffu, ysel, src);
      sdir = __shfl_sync(0xffffffffu, sdir, src);
      if (lane == 0) {
        m = fmin(m, sdir);
        if (ysel < INFINITY) m = fmin(m, s_of_s5(ysel));
        smin[e] = isfinite(m) ? m : 0.0;
      }
      return;
    }
  }
  double m = INFINITY, y = INFINITY;  // direct minimum, minimum of s^5
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (!((cand >> q) & 1u) && !(slo[q] <= shi_min)) continue;
    double v[5];
    float r32;
    if constexpr (f32in) {
      float vf[5];
      if (!load(lane + 32 * q, vf)) continue;
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = widen_f32(vf[k]);
      r32 = vf[0];
    } else {
      if (!load(lane + 32 * q, v)) continue;
      r32 = narrow_f64(v[0]);
    }
    if (!(v[0] > 0.0)) continue;
    const double rr = rcp64(v[0], r32);
    const double p = (gamma - 1.0) * (v[4] - 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) * rr);
    if (!(p > 0.0)) continue;
    if (by5 && s5_in_range(p, rr))
      y = dmin_key(y, s5_of(p, rr));
    else
      m = dmin_key(m, p * pow(v[0], -gamma));
  }
  long long km = dkey(m), ky = dkey(y);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    km = min(km, __shfl_xor_sync(0xffffffffu, km, o));
    ky = min(ky, __shfl_xor_sync(0xffffffffu, ky, o));
  }
  m = dunkey(km);
  y = dunkey(ky);
  if (lane == 0) {
    if (y < INFINITY) m = fmin(m, s_of_s5(y));
    smin[e] = isfinite(m) ? m : 0.0;
  }
}

// Block-wide reductions for the filter kernel.
__device__ __forceinline__ double block_min(double v, double* red) {
  v = warp_min(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = INFINITY;
  for (int i = 0; i < kFilterThreads / 32; ++i) r = fmin(r, red[i]);
  return r;
}

// Order-preserving integer key of a double (signed compare of keys = fmin
// order, positive NaN last), so that minima of doubles reduce on the
// integer pipes instead of the (slow) FP64 pipe.
__device__ __forceinline__ long long dkey(double x) {
  const long long k = __double_as_longlong(x);
  return k ^ ((k >> 63) & 0x7fffffffffffffffLL);
}

__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// exact minima of three doubles over the block (one pair of barriers)
__device__ __forceinline__ void block_min3_key(double& a, double& b, double& c,
                                               long long* red) {
  long long ka = dkey(a), kb = dkey(b), kc = dkey(c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ka = min(ka, __shfl_xor_sync(0xffffffffu, ka, o));
    kb = min(kb, __shfl_xor_sync(0xffffffffu, kb, o));
    kc = min(kc, __shfl_xor_sync(0xffffffffu, kc, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    red[3 * w] = ka;
    red[3 * w + 1] = kb;
    red[3 * w + 2] = kc;
  }
  __syncthreads();
  ka = kb = kc = 0x7fffffffffffffffLL;
  for (int i = 0; i < kFilterThreads / 32; ++i) {
    ka = min(ka, red[3 * i]);
    kb = min(kb, red[3 * i + 1]);
    kc = min(kc, red[3 * i + 2]);
  }
  a = dunkey(ka);
  b = dunkey(kb);
  c = dunkey(kc);
}

// minima of four integer keys over the block (one pair of barriers)
__device__ __forceinline__ void block_min_ll4(long long& a, long long& b, long long& c,
                                              long long& d, long long* red) {
  long long k[4] = {a, b, c, d};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 4; ++i) k[i] = min(k[i], __shfl_xor_sync(0xffffffffu, k[i], o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 4; ++i) red[4 * w + i] = k[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) k[i] = 0x7fffffffffffffffLL;
  for (int j = 0; j < kFilterThreads / 32; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) k[i] = min(k[i], red[4 * j + i]);
  a = k[0];
  b = k[1];
  c = k[2];
  d = k[3];
}

// exact minima of four doubles over the block (one pair of barriers)
__device__ __forceinline__ void block_min4_key(double& a, double& b, double& c, double& d,
                                               long long* red) {
  long long k[4] = {dkey(a), dkey(b), dkey(c), dkey(d)};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 4; ++i) k[i] = min(k[i], __shfl_xor_sync(0xffffffffu, k[i], o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 4; ++i) red[4 * w + i] = k[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) k[i] = 0x7fffffffffffffffLL;
  for (int j = 0; j < kFilterThreads / 32; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) k[i] = min(k[i], red[4 * j + i]);
  a = dunkey(k[0]);
  b = dunkey(k[1]);
  c = dunkey(k[2]);
  d = dunkey(k[3]);
}

// minima of two floats over the block (one pair of barriers)
__device__ __forceinline__ void block_min2f(float& a, float& b, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fminf(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    red[2 * w] = a;
    red[2 * w + 1] = b;
  }
  __syncthreads();
  a = b = INFINITY;
  for (int i = 0; i < kFilterThreads / 32; ++i) {
    a = fminf(a, red[2 * i]);
    b = fminf(b, red[2 * i + 1]);
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < kFilterThreads / 32; ++i) r += red[i];
  return r;
}

__device__ __forceinline__ float silu_f(float x) { return x / (1.0f + __expf(-x)); }

// Predictor evaluated by warp 0 (lane j = hidden unit j); returns z0 on
// lane 0.
static __device__ float mlp_guess(const float feat[4], const __nv_bfloat16* w,
                           const float* norm) {
  const int j = threadIdx.x & 31;
  float xn[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) xn[i] = (feat[i] - norm[i]) / norm[4 + i];
  float a1 = __bfloat162float(w[kB1 + j]);
#pragma unroll
  for (int i = 0; i < 4; ++i) a1 += __bfloat162float(w[kW1 + j * 4 + i]) * xn[i];
  float h1 = silu_f(a1);
  float a2 = __bfloat162float(w[kB2 + j]);
  for (int i = 0; i < kMlpH; ++i)
    a2 += __bfloat162float(w[kW2 + j * kMlpH + i]) * __shfl_sync(0xffffffffu, h1, i);
  float h2 = silu_f(a2);
  float o = __bfloat162float(w[kW3 + j]) * h2;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
  o += __bfloat162float(w[kB3]);
  return o > 20.f ? o : log1pf(__expf(o));
}

// Minima of rho, p and s over a warp's element: slots lane + 32 q of v
// (with their FP32 screens), FP64 values where the screen cannot decide; the
// points of least p and least s^5 selected in double-float arithmetic for
// FP32 values with gamma = 7/5 and computed in FP64 (as k_filter's minima).
// Returns, on every lane, r (exact), p (FP64 at its point), s_dir (minimum
// of s over the points that took the per-point pow) and ys (s^5 at its
// point, FP64).
template <typename T, int NQ, int NP>
__device__ __forceinline__ void warp_minima(const T (&v)[NQ][5], const PtScreen (&sc)[NQ],
                                            double smin, double g, bool by5, dfl gm1d,
                                            double* r_out, double* p_out, double* s_out,
                                            double* ys_out) {
  const int lane = threadIdx.x & 31;
  float phi = INFINITY, shi = INFINITY;
  double rmin = INFINITY;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (lane + 32 * q >= NP) continue;
    rmin = dmin_key(rmin, to_f64(v[q][0]));
    if (sc[q].pos) {
      phi = fminf(phi, sc[q].phi);
      shi = fminf(shi, sc[q].shi);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    phi = fminf(phi, __shfl_xor_sync(0xffffffffu, phi, o));
    shi = fminf(shi, __shfl_xor_sync(0xffffffffu, shi, o));
  }
  double ms = INFINITY;
  long long kp = 0x7fffffffffffffffLL, ky = 0x7fffffffffffffffLL;
  int qp = -1, qy = -1;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (lane + 32 * q >= NP) continue;
    const bool cp = !sc[q].pos || sc[q].plo <= phi;
    const bool cs = smin > 0.0 && (!sc[q].pos || sc[q].slo <= shi);
    if (!cp && !cs) continue;
    double pk = 0.0, yk = 0.0;
    bool ykey = false, exact = true;
    if constexpr (sizeof(T) == 4) {
      const float r = v[q][0];
      if (by5 && r >= 0x1p-100f && r <= 0x1p100f) {
        bool amb;
        const dfl rr = df_rcp(r);
        const dfl pd = df_pressure(v[q][1], v[q][2], v[q][3], v[q][4], rr, gm1d, &amb);
        if (!amb) {
          exact = false;
          pk = df_to_f64(pd);
          if (cs) {
            if (df_s5_key(pd, rr, &yk)) {
              ykey = true;
            } else {
              double w[5];
#pragma unroll
              for (int k = 0; k < 5; ++k) w[k] = to_f64(v[q][k]);
              ms = dmin_key(ms, pressure64(w, g) * pow(w[0], -g));
            }
          }
        }
      }
    }
    if (exact) {
      double w[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) w[k] = to_f64(v[q][k]);
      const bool rpos = w[0] > 0.0;
      const double rr64 = rpos ? rcp64(w[0], sizeof(T) == 4 ? float(v[q][0]) : narrow_f64(w[0])) : 0.0;
      pk = rpos ? (g - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) * rr64)
                : pressure64(w, g);
      if (cs) {
        if (!rpos) {
          ms = -INFINITY;
        } else if (by5 && s5_in_range(pk, rr64)) {
          yk = s5_of(pk, rr64);
          ykey = true;
        } else {
          ms = dmin_key(ms, pk * pow(w[0], -g));
        }
      }
    }
    const bool pnan = (__double_as_longlong(pk) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
    const long long kt = (dkey(pk) & ~0x1fLL) | lane;
    if (cp && !pnan && kt < kp) {
      kp = kt;
      qp = q;
    }
    if (ykey) {
      const long long kyt = (dkey(yk) & ~0x1fLL) | lane;
      if (kyt < ky) {
        ky = kyt;
        qy = q;
      }
    }
  }
  long long kr = dkey(rmin), kms = dkey(ms), kpm = kp, kym = ky;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kr = min(kr, __shfl_xor_sync(0xffffffffu, kr, o));
    kms = min(kms, __shfl_xor_sync(0xffffffffu, kms, o));
    kpm = min(kpm, __shfl_xor_sync(0xffffffffu, kpm, o));
    kym = min(kym, __shfl_xor_sync(0xffffffffu, kym, o));
  }
  // the selected points' FP64 values, from their lanes
  double psel = INFINITY, ysel = INFINITY, sdir = INFINITY;
  if (qp >= 0 && kp == kpm) {
    double w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = to_f64(v[qp][k]);
    psel = pressure64(w, g);
  }
  if (qy >= 0 && ky == kym) {
    double w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = to_f64(v[qy][k]);
    const double rr64 = rcp64(w[0], sizeof(T) == 4 ? float(v[qy][0]) : narrow_f64(w[0]));
    const double p64 = (g - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) * rr64);
    if (s5_in_range(p64, rr64)) ysel = s5_of(p64, rr64);
    else sdir = p64 * pow(w[0], -g);
  }
  const bool hp = kpm != 0x7fffffffffffffffLL, hy = kym != 0x7fffffffffffffffLL;
  psel = __shfl_sync(0xffffffffu, psel, hp ? int(kpm & 0x1f) : 0);
  ysel = __shfl_sync(0xffffffffu, ysel, hy ? int(kym & 0x1f) : 0);
  sdir = __shfl_sync(0xffffffffu, sdir, hy ? int(kym & 0x1f) : 0);
  *r_out = dunkey(kr);
  *p_out = hp ? psel : INFINITY;
  *s_out = fmin(dunkey(kms), hy ? sdir : INFINITY);
  *ys_out = hy ? ysel : INFINITY;
}

// The zeta = 0 test of every element of a type, one warp per element, on
// the stage value (reg / regR) at the solution points and its flux-point
// traces (uf, from the volume kernel): elements that meet the constraints
// are left alone (zeta 0, one evaluation); the others are listed for
// k_filter, which takes the oracle's modal form from there.
template <typename T, typename TR, int NU, int NF>
__global__ void k_filter_check(long long ne, const T* __restrict__ reg,
                               const TR* __restrict__ regR, const T* __restrict__ uf,
                               FilterArgs fa, int32_t* __restrict__ list,
                               int* __restrict__ count) {
  constexpr int NP = NU + NF, NQ = (NP + 31) / 32;
  const int lane = threadIdx.x & 31;
  const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= ne) return;  // whole warps
  const double g = fa.gamma;
  const float gf = float(g);
  const bool by5 = entropy_by_s5(g);
  const float gm1h = float(g - 1.0);
  const dfl gm1d{gm1h, float((g - 1.0) - widen_f32(gm1h))};
  const double smin = fa.smin[e];
  const double sb = smin * (1.0 - fa.tau);
  T v[NQ][5];
  PtScreen sc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = lane + 32 * q;
    sc[q].pos = false;
    sc[q].plo = sc[q].slo = INFINITY;
#pragma unroll
    for (int k = 0; k < 5; ++k) v[q][k] = T(0);
    if (i >= NP) continue;
#pragma unroll
    for (int k = 0; k < 5; ++k)
      v[q][k] = i < NU ? (reg ? reg[(e * 5 + k) * NU + i] : T(regR[(e * 5 + k) * NU + i]))
                       : uf[(e * 5 + k) * NF + (i - NU)];
    sc[q] = screen_point(float(v[q][0]), float(v[q][1]), float(v[q][2]), float(v[q][3]),
                         float(v[q][4]), gf);
  }
  double r, p, sdir, ys;
  warp_minima<T, NQ, NP>(v, sc, smin, g, by5, gm1d, &r, &p, &sdir, &ys);
  if (lane != 0) return;
  double s_term = INFINITY;
  if (smin > 0.0) {
    const double sb2 = sb * sb, sb5 = sb2 * sb2 * sb;
    s_term = (sdir >= sb && !(ys < sb5)) ? 0.0 : -1.0;
  }
  const double gm = fmin(r - kEpsPos, fmin(p - kEpsPos, s_term));
  if (!isnan(gm) && gm >= 0.0) {
    if (fa.zeta_last) {
      fa.zeta_last[e] = 0.f;
      fa.evals_last[e] = 1;
    }
  } else {
    list[atomicAdd(count, 1)] = int32_t(e);
  }
}

// the five values of one mode of ush (a 16-byte aligned row of 8): one
// 128-bit and one 32-bit shared load in FP32
__device__ __forceinline__ void get_modes5(const float (&r)[8], float (&a)[5]) {
  const float4 x = *reinterpret_cast<const float4*>(&r[0]);
  a[0] = x.x;
  a[1] = x.y;
  a[2] = x.z;
  a[3] = x.w;
  a[4] = r[4];
}
__device__ __forceinline__ void get_modes5(const double (&r)[8], double (&a)[5]) {
  const double2 x = *reinterpret_cast<const double2*>(&r[0]);
  const double2 y = *reinterpret_cast<const double2*>(&r[2]);
  a[0] = x.x;
  a[1] = x.y;
  a[2] = y.x;
  a[3] = y.y;
  a[4] = r[4];
}

// Filter the stage value of each element that violates the constraints.
// reg / regR: the register holding the new stage value (type T or TR, one
// of them null); uf: this type's flux-point traces of that value.
template <typename T, typename TR, int NU, int NF>
__global__ void __launch_bounds__(kFilterThreads)
    k_filter(long long ne, T* __restrict__ reg, TR* __restrict__ regR,
             T* __restrict__ uf, FilterOps<T> op, FilterArgs fa,
             const int32_t* __restrict__ list, const int* __restrict__ count) {
  constexpr int NM = NU, NP = NU + NF;
  __shared__ T uh[5][NM];       // modal coefficients
  __shared__ __align__(16) T ush[NM][8];  // sigma_k u^_k of an evaluation (5 used)
  __shared__ double red[kFilterThreads / 32];
  __shared__ long long redk[4 * (kFilterThreads / 32)];
  __shared__ float redf[2 * (kFilterThreads / 32)];
  __shared__ double s_z;        // requested strength
  // CTA b filters element list[b] of the k_filter_check list
  if (int(blockIdx.x) >= *count) return;
  const long long e = list[blockIdx.x];
  const int tid = threadIdx.x;
  if (e >= ne) return;
  const double g = fa.gamma;
  const float gf = float(g);
  const bool by5 = entropy_by_s5(g);
  const float gm1h = float(g - 1.0);
  const dfl gm1d{gm1h, float((g - 1.0) - widen_f32(gm1h))};  // gamma - 1, double-float
  __shared__ double s_sel[3];  // FP64 values at the selected points
  __shared__ T us[5][NU];
  const double smin = fa.smin[e];
  const double sb = smin * (1.0 - fa.tau);
  // Exact minima of rho, p and s = p rho^-g (-inf where rho <= 0) of the
  // filtered polynomial at strength z over the solution and flux points
  // (all threads).  Every point is screened in FP32 (screen_point); the FP64
  // p and s are computed only for the points whose lower bound reaches the
  // block's smallest upper bound, so the minima equal those of an all-FP64
  // pass over the same values.
  constexpr int NPT = (NP + kFilterThreads - 1) / kFilterThreads;
  struct Mins {
    double r, p, s;  // s: minimum over the points that took the per-point pow
    double ys;       // minimum of s^5 over the others (entropy_by_s5)
  };
  // the entropy minimum of an evaluation (one pow, by the thread that needs it)
  auto smin_of = [](const Mins& q) -> double {
    return q.ys < INFINITY ? fmin(q.s, s_of_s5(q.ys)) : q.s;
  };
  auto minima = [&](double z) -> Mins {
    for (int m = tid; m < NM; m += kFilterThreads) {
      double d = double(op.deg[m]);
      const T sk = sizeof(T) == 4 ? T(__expf(-float(z * d * d))) : T(exp(-z * d * d));
#pragma unroll
      for (int k = 0; k < 5; ++k) ush[m][k] = sk * uh[k][m];
    }
    __syncthreads();
    T v[NPT][5];
    PtScreen sc[NPT];
    T rmin_t = T(INFINITY);
    float phi = INFINITY, shi = INFINITY;
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      const int i = tid + q * kFilterThreads;
#pragma unroll
      for (int k = 0; k < 5; ++k) v[q][k] = T(0);
      sc[q].pos = false;
      sc[q].plo = sc[q].slo = INFINITY;  // no point: never a candidate
      if (i >= NP) continue;
      for (int m = 0; m < NM; ++m) {
        const T w = op.VT[m * NP + i];
        T a[5];
        get_modes5(ush[m], a);
#pragma unroll
        for (int k = 0; k < 5; ++k) v[q][k] += w * a[k];
      }
      rmin_t = sizeof(T) == 4 ? T(fminf(float(rmin_t), float(v[q][0])))
                              : T(fmin(double(rmin_t), double(v[q][0])));
      sc[q] = screen_point(float(v[q][0]), float(v[q][1]), float(v[q][2]),
                           float(v[q][3]), float(v[q][4]), gf);
      if (sc[q].pos) {
        phi = fminf(phi, sc[q].phi);
        shi = fminf(shi, sc[q].shi);
      }
    }
    block_min2f(phi, shi, redf);
    double rmin = double(rmin_t), mp = INFINITY, ms = INFINITY, ys = INFINITY;
    if constexpr (sizeof(T) == 4) {
      if (by5) {
        // FP32 values, gamma = 7/5: the points of least p and of least s
        // are selected in double-float arithmetic (~2^-43; FP64 only where
        // its pressure is too close to zero to sign), then p and s^5 are
        // computed in FP64 at the selected points.  Keys carry the thread
        // in their low bits, so the selected point is unique.
        long long kp = 0x7fffffffffffffffLL, ky = 0x7fffffffffffffffLL;
        int qp = -1, qy = -1;
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
          if (tid + q * kFilterThreads >= NP) continue;
          const bool cp = !sc[q].pos || sc[q].plo <= phi;
          const bool cs = smin > 0.0 && (!sc[q].pos || sc[q].slo <= shi);
          if (!cp && !cs) continue;
          const float r = float(v[q][0]);
          bool amb = !(r >= 0x1p-100f && r <= 0x1p100f);
          dfl rr{0.f, 0.f}, pd{0.f, 0.f};
          if (!amb) {
            rr = df_rcp(r);
            pd = df_pressure(float(v[q][1]), float(v[q][2]), float(v[q][3]),
                             float(v[q][4]), rr, gm1d, &amb);
          }
          double pk, yk;
          bool ykey = false;
          if (amb) {  // FP64 at this point
            double w[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) w[k] = to_f64(v[q][k]);
            pk = pressure64(w, g);
            if (cs) {
              if (!(w[0] > 0.0)) {
                ms = -INFINITY;
              } else {
                const double rr64 = rcp64(w[0], r);
                if (s5_in_range(pk, rr64)) {
                  yk = s5_of(pk, rr64);
                  ykey = true;
                } else {
                  ms = dmin_key(ms, pk * pow(w[0], -g));
                }
              }
            }
          } else {
            pk = df_to_f64(pd);
            if (cs) {
              if (df_s5_key(pd, rr, &yk)) {
                ykey = true;
              } else {
                double w[5];
#pragma unroll
                for (int k = 0; k < 5; ++k) w[k] = to_f64(v[q][k]);
                ms = dmin_key(ms, pressure64(w, g) * pow(w[0], -g));
              }
            }
          }
          const bool pnan = (__double_as_longlong(pk) & 0x7fffffffffffffffLL) >
                            0x7ff0000000000000LL;  // ignored, like fmin
          const long long kt = (dkey(pk) & ~0xffLL) | tid;
          if (cp && !pnan && kt < kp) {
            kp = kt;
            qp = q;
          }
          if (ykey) {
            const long long kyt = (dkey(yk) & ~0xffLL) | tid;
            if (kyt < ky) {
              ky = kyt;
              qy = q;
            }
          }
        }
        long long kr = dkey(rmin), kms = dkey(ms), kpm = kp, kym = ky;
        block_min_ll4(kr, kpm, kms, kym, redk);
        rmin = dunkey(kr);
        ms = dunkey(kms);
        // the selected points' FP64 values (one writer each)
        if (qp >= 0 && kp == kpm) {
          double w[5];
#pragma unroll
          for (int k = 0; k < 5; ++k) w[k] = to_f64(v[qp][k]);
          s_sel[0] = pressure64(w, g);
        }
        if (qy >= 0 && ky == kym) {
          double w[5];
#pragma unroll
          for (int k = 0; k < 5; ++k) w[k] = to_f64(v[qy][k]);
          const double rr64 = rcp64(w[0], float(v[qy][0]));
          const double p64 = (g - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) * rr64);
          s_sel[1] = s5_in_range(p64, rr64) ? s5_of(p64, rr64) : INFINITY;
          if (!s5_in_range(p64, rr64)) s_sel[2] = p64 * pow(w[0], -g);
        }
        __syncthreads();
        mp = kpm == 0x7fffffffffffffffLL ? INFINITY : s_sel[0];
        ys = kym == 0x7fffffffffffffffLL ? INFINITY : s_sel[1];
        if (kym != 0x7fffffffffffffffLL && !(s_sel[1] < INFINITY)) ms = fmin(ms, s_sel[2]);
        // (s_sel is written again only after the next evaluation's barriers)
        return Mins{rmin, mp, ms, ys};
      }
    }
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
      if (tid + q * kFilterThreads >= NP) continue;
      const bool cp = !sc[q].pos || sc[q].plo <= phi;
      const bool cs = smin > 0.0 && (!sc[q].pos || sc[q].slo <= shi);
      if (!cp && !cs) continue;
      double w[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) w[k] = to_f64(v[q][k]);
      // one FP64 reciprocal per point (Newton steps from FP32, rcp64): 1/rho
      // serves p and the s^5 key
      const bool rpos = w[0] > 0.0;
      const double rr =
          rpos ? rcp64(w[0], sizeof(T) == 4 ? float(v[q][0]) : narrow_f64(w[0])) : 0.0;
      const double p =
          rpos ? (g - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) * rr)
               : pressure64(w, g);
      if (cp) mp = dmin_key(mp, p);
      if (cs) {
        if (!rpos)
          ms = -INFINITY;
        else if (by5 && s5_in_range(p, rr))
          ys = dmin_key(ys, s5_of(p, rr));
        else
          ms = dmin_key(ms, p * pow(w[0], -g));
      }
    }
    block_min4_key(rmin, mp, ms, ys, redk);
    return Mins{rmin, mp, ms, ys};
  };
  // unfiltered state admissible (the sign of the margin below, which the
  // positive means do not change): nothing to do (uniform across the block).
  // The entropy term's sign without a pow: s >= sb <=> s^5 >= sb^5.
  auto admissible = [&](const Mins& q) -> bool {
    double s_term = INFINITY;
    if (smin > 0.0) {
      const double sb2 = sb * sb, sb5 = sb2 * sb2 * sb;
      s_term = (q.s >= sb && !(q.ys < sb5)) ? 0.0 : -1.0;
    }
    const double gm = fmin(q.r - kEpsPos, fmin(q.p - kEpsPos, s_term));
    return !isnan(gm) && gm >= 0.0;
  };
  auto leave_unfiltered = [&]() {
    if (tid == 0 && fa.zeta_last) {
      fa.zeta_last[e] = 0.f;
      fa.evals_last[e] = 1;
    }
  };
  // (k_filter_check left the elements that pass at zeta = 0 on the stage
  // value and its traces alone)
  // modal coefficients u^ = V^-1 u
  for (int z = tid; z < NU; z += kFilterThreads)
#pragma unroll
    for (int k = 0; k < 5; ++k)
      us[k][z] = reg ? reg[(e * 5 + k) * NU + z] : T(regR[(e * 5 + k) * NU + z]);
  __syncthreads();
  for (int m = tid; m < NM; m += kFilterThreads) {
    T acc[5] = {0, 0, 0, 0, 0};
    for (int z = 0; z < NU; ++z) {
      T w = op.VinvT[z * NM + m];
#pragma unroll
      for (int k = 0; k < 5; ++k) acc[k] += w * us[k][z];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) uh[k][m] = acc[k];
  }
  // the same test on the modal evaluation (the oracle's form)
  Mins m0 = minima(0.0);
  if (admissible(m0)) {
    leave_unfiltered();
    return;
  }
  // a filtered element: its entropy minimum at z = 0 (one pow, warp 0:
  // the predictor's features and thread 0's margin read it)
  if (tid < 32) m0.s = smin_of(m0);
  m0.ys = INFINITY;
  // element means of density and pressure (normalise the margin)
  double wr = 0.0, wp = 0.0, ws = 0.0;
  for (int z = tid; z < NU; z += kFilterThreads) {
    const double w5[5] = {double(us[0][z]), double(us[1][z]), double(us[2][z]),
                          double(us[3][z]), double(us[4][z])};
    const double p = pressure64(w5, g);
    double w = double(op.W[z]);
    wr += w * double(us[0][z]);
    wp += w * p;
    ws += w;
  }
  const double wsum = block_sum(ws, red);
  const double rmean = fmax(block_sum(wr, red) / wsum, kEpsPos);
  const double pmean = fmax(block_sum(wp, red) / wsum, kEpsPos);
  // margin g(z) = min((rho-eps)/rho_mean, (p-eps)/p_mean, (s-sb)/s_min)
  auto gval = [&](const Mins& q) -> double {
    const double gr = (q.r - kEpsPos) / rmean, gp = (q.p - kEpsPos) / pmean;
    const double gs = smin > 0.0 ? (smin_of(q) - sb) / smin : INFINITY;
    double gm = fmin(gr, fmin(gp, gs));
    if (isnan(gm)) gm = -INFINITY;
    return gm;
  };
  auto margin = [&](double z) -> double { return gval(minima(z)); };
  // predictor inputs from the unfiltered state (z = 0)
  float feat[4] = {0.f, 0.f, 0.f, 0.f};
  if (fa.mlp || fa.samples) {
    double eh = 0.0, et = 0.0;
    for (int m = tid; m < NM; m += kFilterThreads) {
      double d = double(op.deg[m]), c = double(uh[0][m]);
      if (d > 1.0) eh += c * c;
      if (d > 0.0) et += c * c;
    }
    eh = block_sum(eh, red);
    et = block_sum(et, red);
    feat[0] = float(fmin(fmax(log10((eh + 1e-30) / (et + 1e-30)), -30.0), 30.0));
    feat[1] = float(fmin(fmax(m0.r / rmean, -30.0), 30.0));
    feat[2] = float(fmin(fmax(m0.p / pmean, -30.0), 30.0));
    // log10 of the entropy-bound violation (floor 1e-14)
    double f3 = 1.0;
    if (smin > 0.0 && m0.s > -INFINITY && m0.r > 0.0 && m0.p > 0.0)
      f3 = fmax((smin - m0.s) / smin, 1e-14);
    feat[3] = float(log10(f3));
  }
  const double g0 = gval(m0);
  // ---- root-find.  Thread 0 runs the bracketing and Illinois logic as a
  // state machine and publishes the next strength in shared memory; every
  // evaluation of the margin is a block operation.
  enum { kPlainHi = 0, kGuess = 1, kDown = 2, kUp = 3, kIllinois = 4, kDone = 5 };
  __shared__ double s_next;
  __shared__ int s_go;
  // ghr: the margin at hi (ghi is halved by the Illinois rule)
  double lo = 0.0, glo = g0, hi = kZetaMax, ghi = 0.0, ghr = 0.0, result = 0.0, zc = 0.0;
  int evals = 1, state = kPlainHi, it = 0, side = 0;
  bool fallback = false, use_guess = false;
  if (fa.mlp) {
    float z0 = 0.f;
    if (tid < 32) z0 = mlp_guess(feat, fa.mlp, fa.mlp_norm);
    if (tid == 0) s_z = double(z0);
    __syncthreads();
    const double guess = s_z;
    use_guess = guess > 0.0 && guess < kZetaMax;
    if (use_guess) {
      state = kGuess;
      zc = guess;
    }
  }
  if (state == kPlainHi) zc = kZetaMax;
  // next Illinois point, or kDone when the feasible end's margin is within
  // tau, the bracket is tight or the evaluations are spent
  auto illinois_next = [&]() {
    if (!(ghr > fa.tau && hi - lo > kRelTol * hi && evals < kMaxEvals)) {
      state = kDone;
      result = hi;
      return;
    }
    double z = (lo * ghi - hi * glo) / (ghi - glo);
    if (!(lo < z && z < hi)) z = 0.5 * (lo + hi);
    zc = z;
  };
  if (tid == 0) {
    s_next = zc;
    s_go = 1;
  }
  for (;;) {
    __syncthreads();
    if (!s_go) break;
    const double z = s_next;
    const Mins mz = minima(z);  // ends with a barrier: s_next / s_go reusable
    if (tid != 0) continue;
    const double gz = gval(mz);
    ++evals;
    switch (state) {
      case kPlainHi:
        ghi = ghr = gz;
        if (gz < 0.0) {
          state = kDone;
          fallback = true;
          result = kZetaMax;
        } else {
          state = kIllinois;
          illinois_next();
        }
        break;
      case kGuess:
        if (gz >= 0.0) {
          hi = z;
          ghi = ghr = gz;
          state = kDown;
          zc = z / fa.ratio;
          if (gz <= fa.tau) {
            state = kDone;
            result = hi;
          }
        } else {
          lo = z;
          glo = gz;
          state = kUp;
          zc = fmin(fa.ratio * z, kZetaMax);
        }
        it = 0;
        break;
      case kDown:  // halve until the margin is negative
        if (gz < 0.0) {
          lo = z;
          glo = gz;
          state = kIllinois;
          illinois_next();
        } else {
          hi = z;
          ghi = ghr = gz;
          if (z < 1e-6 || gz <= fa.tau) {
            state = kDone;
            result = hi;
          } else {
            zc = 0.5 * z;
            if (++it >= 64) {
              state = kDone;
              fallback = true;
              result = kZetaMax;
            }
          }
        }
        break;
      case kUp:  // double until the margin is non-negative
        if (gz >= 0.0) {
          hi = z;
          ghi = ghr = gz;
          state = kIllinois;
          illinois_next();
        } else {
          lo = z;
          glo = gz;
          if (z >= kZetaMax) {
            state = kDone;
            fallback = true;
            result = kZetaMax;
          } else {
            zc = fmin(2.0 * z, kZetaMax);
            if (++it >= 64) {
              state = kDone;
              fallback = true;
              result = kZetaMax;
            }
          }
        }
        break;
      case kIllinois:
        if (gz >= 0.0) {
          hi = z;
          ghi = ghr = gz;
          if (side == 1) glo *= 0.5;
          side = 1;
        } else {
          lo = z;
          glo = gz;
          if (side == -1) ghi *= 0.5;
          side = -1;
        }
        illinois_next();
        break;
    }
    s_go = state != kDone;
    s_next = state == kDone ? result : zc;
  }
  // every thread: the strength found by thread 0
  result = s_next;
  // write the filtered state and its flux-point values
  for (int m = tid; m < NM; m += kFilterThreads) {
    const T sk = T(exp(-result * double(op.deg[m]) * double(op.deg[m])));
#pragma unroll
    for (int k = 0; k < 5; ++k) ush[m][k] = sk * uh[k][m];
  }
  __syncthreads();
  for (int i = tid; i < NP; i += kFilterThreads) {
    T v[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < NM; ++m) {
      const T w = op.VT[m * NP + i];
      T a[5];
      get_modes5(ush[m], a);
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] += w * a[k];
    }
    if (i < NU) {
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        if (reg) reg[(e * 5 + k) * NU + i] = v[k];
        else regR[(e * 5 + k) * NU + i] = TR(v[k]);
      }
    } else {
      int f = i - NU;
#pragma unroll
      for (int k = 0; k < 5; ++k) uf[(e * 5 + k) * NF + f] = v[k];
    }
  }
  if (tid == 0) {
    if (fa.zeta_last) {
      fa.zeta_last[e] = float(result);
      fa.evals_last[e] = evals;
    }
    atomicAdd(&fa.stats->filtered, 1ull);
    atomicAdd(&fa.stats->evals, (unsigned long long)evals);
    if (fallback) atomicAdd(&fa.stats->fallbacks, 1ull);
    if (use_guess) atomicAdd(&fa.stats->guessed, 1ull);
    if (!fallback && fa.samples) {
      unsigned long long i = atomicAdd(&fa.stats->samples, 1ull);
      if (i < fa.cap) {
#pragma unroll
        for (int k = 0; k < 4; ++k) fa.samples[i * 5 + k] = feat[k];
        fa.samples[i * 5 + 4] = float(result);
      }
    }
  }
}

// ------------------------------------------------------------------ MLP
// Training is deterministic: one kernel computes per-sample activations and
// deltas, a second reduces every parameter's gradient over all samples in a
// fixed order, a third applies Adam.

__device__ __forceinline__ float dsilu_f(float x) {
  float s = 1.0f / (1.0f + expf(-x));
  return s * (1.0f + x * (1.0f - s));
}

// per sample: xn[4], h1[32], h2[32], da1[32], da2[32], do, loss term
constexpr int kMlpScratch = 4 + 32 * 4 + 2;

static __global__ void k_mlp_sample(int n, const float* __restrict__ w,
                             const float* __restrict__ x,
                             const float* __restrict__ zstar,
                             float* __restrict__ scr) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float* o = scr + size_t(s) * kMlpScratch;
  float xn[4], a1[32], h1[32], a2[32], h2[32];
  for (int i = 0; i < 4; ++i) xn[i] = (x[s * 4 + i] - w[kMean + i]) / w[kStd + i];
  for (int j = 0; j < 32; ++j) {
    float a = w[kB1 + j];
    for (int i = 0; i < 4; ++i) a += w[kW1 + j * 4 + i] * xn[i];
    a1[j] = a;
    h1[j] = a / (1.0f + expf(-a));
  }
  float out = w[kB3];
  for (int j = 0; j < 32; ++j) {
    float a = w[kB2 + j];
    for (int i = 0; i < 32; ++i) a += w[kW2 + j * 32 + i] * h1[i];
    a2[j] = a;
    h2[j] = a / (1.0f + expf(-a));
    out += w[kW3 + j] * h2[j];
  }
  float z0 = out > 20.f ? out : log1pf(expf(out));
  float r = logf(z0) - logf(zstar[s]);
  float dz0 = 2.0f * r / float(n) / z0;
  float dout = dz0 / (1.0f + expf(-out));
  float da2[32];
  for (int j = 0; j < 32; ++j) da2[j] = dout * w[kW3 + j] * dsilu_f(a2[j]);
  for (int i = 0; i < 4; ++i) o[i] = xn[i];
  for (int i = 0; i < 32; ++i) {
    float dh1 = 0.f;
    for (int j = 0; j < 32; ++j) dh1 += da2[j] * w[kW2 + j * 32 + i];
    o[4 + i] = h1[i];
    o[36 + i] = h2[i];
    o[68 + i] = dh1 * dsilu_f(a1[i]);
    o[100 + i] = da2[i];
  }
  o[132] = dout;
  o[133] = r * r / float(n);
}

// one thread per trainable parameter (and one for the loss), summing over
// samples in order
static __global__ void k_mlp_reduce(int n, const float* __restrict__ scr,
                             float* __restrict__ grad, float* __restrict__ loss) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > kMlpTrain) return;
  double acc = 0.0;
  for (int s = 0; s < n; ++s) {
    const float* o = scr + size_t(s) * kMlpScratch;
    float v;
    if (q == kMlpTrain) v = o[133];
    else if (q < kB1) v = o[68 + q / 4] * o[q % 4];                  // W1
    else if (q < kW2) v = o[68 + (q - kB1)];                         // b1
    else if (q < kB2) {                                              // W2
      int r = q - kW2;
      v = o[100 + r / 32] * o[4 + r % 32];
    } else if (q < kW3) v = o[100 + (q - kB2)];                      // b2
    else if (q < kB3) v = o[132] * o[36 + (q - kW3)];                // W3
    else v = o[132];                                                 // b3
    acc += double(v);
  }
  if (q == kMlpTrain) *loss = float(acc);
  else grad[q] = float(acc);
}

static __global__ void k_mlp_adam(float* __restrict__ w, const float* __restrict__ grad,
                           float* __restrict__ m1, float* __restrict__ m2,
                           int step, float lr) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kMlpTrain) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float gq = grad[q];
  float a = b1 * m1[q] + (1 - b1) * gq;
  float b = b2 * m2[q] + (1 - b2) * gq * gq;
  m1[q] = a;
  m2[q] = b;
  float ah = a / (1 - powf(b1, float(step)));
  float bh = b / (1 - powf(b2, float(step)));
  w[q] -= lr * ah / (sqrtf(bh) + eps);
}

}  // namespace frgb
