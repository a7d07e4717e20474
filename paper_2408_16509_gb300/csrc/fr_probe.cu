// Arithmetic throughput probe: the peak that bounds the FP64 right-hand side
// on this GPU (its FP64 units, not its memory, limit the plain FP64 form).
// A measurement aid for the roofline of the library's kernels; the paper has
// no counterpart.  See include/frgb.h (fr_probe_fma).
#include <cuda_runtime.h>

#include <string>

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

}  // namespace

extern "C" int fr_probe_fma(int device, int dtype, int64_t iters, double* ms,
                            double* flops) {
  if (!ms || !flops) return fail(FR_EINVAL, "null argument");
  if (iters < 1) return fail(FR_EINVAL, "iters must be positive");
  if (dtype != FR_DTYPE_F64 && dtype != FR_DTYPE_F32) return fail(FR_EINVAL, "unknown dtype");
  CK(cudaSetDevice(device));
  return dtype == FR_DTYPE_F64 ? run_probe<double>(device, iters, ms, flops)
                               : run_probe<float>(device, iters, ms, flops);
}
