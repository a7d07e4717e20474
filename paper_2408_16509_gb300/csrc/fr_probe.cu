// Arithmetic throughput probe: the peak that bounds the FP64 right-hand side
// on this GPU (its FP64 units, not its memory, limit the plain FP64 form).
// A measurement aid for the roofline of the library's kernels; the paper has
// no counterpart.  See include/frgb.h (fr_probe_fma).
#include <cuda_runtime.h>

#include <string>

#include "fr_convert.cuh"
#include "fr_err.hpp"

using namespace frgb;

namespace {

// Eight independent FMA chains per thread (enough to cover the FMA latency
// at a few warps per scheduler); the results are stored so nothing is
// eliminated.  Flops per launch: 2 * 8 * iters * threads.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(long long iters, T a, T b, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run_probe(int device, long long iters, double* ms, double* flops) {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int threads = 256, blocks = sms * 8;
  T* out = nullptr;
  CK(cudaMalloc(&out, size_t(blocks) * threads * sizeof(T)));
  cudaStream_t s;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a = 1 - 2^-20, b = 2^-20: the chains stay bounded and finite
  const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1048576.0);
  k_fma_probe<T><<<blocks, threads, 0, s>>>(iters / 16 + 1, a, b, out);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_probe<T><<<blocks, threads, 0, s>>>(iters, a, b, out);
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(out);
  if (err != cudaSuccess) return fail(FR_ECUDA, std::string("probe: ") + cudaGetErrorString(err));
  *ms = t;
  *flops = 2.0 * 8.0 * double(iters) * double(blocks) * threads;
  return FR_OK;
}

// splitmix64 (Steele, Lea & Flood 2014): the test patterns of the
// conversion check, one counter per pattern.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Pattern i: a random 32-bit float pattern for widening, and a 64-bit double
// pattern for narrowing drawn from one of four classes: any bits, exponents
// near the float range (with random sign and fraction), exact ties of the
// dropped 29 bits, and all-ones fractions at the top and bottom exponents
// (carries into the exponent and out of the range).
__global__ void k_convert_check(unsigned long long seed, long long n,
                                unsigned long long* bad) {
  unsigned long long nb = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long r = mix64(seed ^ mix64((unsigned long long)i));
    const unsigned long long q = mix64(r);
    const float f = __uint_as_float(uint32_t(r));
    const double w0 = double(f), w1 = widen_f32(f);
    const bool wnan = w0 != w0;
    if (wnan ? (w1 == w1) : (__double_as_longlong(w0) != __double_as_longlong(w1))) ++nb;
    unsigned long long d = q;
    const unsigned long long sign = q & 0x8000000000000000ull;
    const unsigned long long frac = q & 0xfffffffffffffull;
    switch (int(r >> 62)) {
      case 0: break;
      case 1: d = sign | ((unsigned long long)(860 + (r >> 32) % 330) << 52) | frac; break;
      case 2:
        d = sign | ((unsigned long long)(890 + (r >> 32) % 270) << 52) |
            (frac & ~0x1fffffffull) | 0x10000000ull;
        break;
      default: {
        const int k = int((r >> 32) % 6);  // exponents 895-897 and 1149-1151
        d = sign | ((unsigned long long)(k < 3 ? 895 + k : 1146 + k) << 52) |
            ((r >> 40) & 1 ? 0xfffffffffffffull : (frac | 0xfffffe0000000ull));
      }
    }
    const double dv = __longlong_as_double((long long)d);
    const float n0 = __double2float_rn(dv), n1 = narrow_f64(dv);
    const bool nnan = n0 != n0;
    if (nnan ? (n1 == n1) : (__float_as_uint(n0) != __float_as_uint(n1))) ++nb;
    // the FP64 reciprocal, positive x across and beyond its fast range:
    // within 2 units in the last place of the division
    const double x = fabs(dv);
    if (x > 0.0 && x < INFINITY) {
      const double r0 = 1.0 / x, r1 = rcp64(x, __double2float_rn(x));
      const long long u = __double_as_longlong(r0) - __double_as_longlong(r1);
      if (r0 > 0.0 && r0 < INFINITY && (u > 2 || u < -2)) ++nb;
      // the fifth root: r^5 = x to 5e-15 relative (r within about 2 units
      // in the last place; the FP64 fifth power adds ~4 roundings).  pow(x,
      // 0.2) is no reference here: 0.2 is 1/5 only to 1e-17, which moves
      // the result by 1e-17 |ln x| relative (8e-15 at x = 1e300)
      const double q = root5(x);
      const double q2 = q * q, q5 = q2 * q2 * q;
      if (x >= 1e-290 && x <= 1e290 && !(fabs(q5 - x) <= 5e-15 * x)) ++nb;
    }
  }
  if (nb) atomicAdd(bad, nb);
}

}  // namespace

extern "C" int fr_check_conversions(int device, uint64_t seed, int64_t n,
                                    int64_t* mismatches) {
  if (!mismatches) return fail(FR_EINVAL, "null argument");
  if (n < 0) return fail(FR_EINVAL, "n must not be negative");
  CK(cudaSetDevice(device));
  unsigned long long* bad = nullptr;
  CK(cudaMalloc(&bad, sizeof(unsigned long long)));
  unsigned long long h = 0;
  cudaError_t err = cudaMemset(bad, 0, sizeof(h));
  if (err == cudaSuccess && n > 0) {
    k_convert_check<<<1024, 256>>>(seed, n, bad);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaMemcpy(&h, bad, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(bad);
  if (err != cudaSuccess) return fail(FR_ECUDA, std::string("conversion check: ") + cudaGetErrorString(err));
  *mismatches = int64_t(h);
  return FR_OK;
}

extern "C" int fr_probe_fma(int device, int dtype, int64_t iters, double* ms,
                            double* flops) {
  if (!ms || !flops) return fail(FR_EINVAL, "null argument");
  if (iters < 1) return fail(FR_EINVAL, "iters must be positive");
  if (dtype != FR_DTYPE_F64 && dtype != FR_DTYPE_F32) return fail(FR_EINVAL, "unknown dtype");
  CK(cudaSetDevice(device));
  return dtype == FR_DTYPE_F64 ? run_probe<double>(device, iters, ms, flops)
                               : run_probe<float>(device, iters, ms, flops);
}
