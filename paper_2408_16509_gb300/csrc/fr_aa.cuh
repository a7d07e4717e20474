// Anti-aliased transformed flux (Section 3.2, "Anti-aliasing").
//
// Instead of collocating f~ = S F(u) at the solution points, the flux is
// taken at the points x_q of a volume rule of degree qdeg and projected onto
// the solution space by least squares:
//     u_q = B u,  (grad u)_q = B grad u,  f~_q = S(x_q) F(u_q, (grad u)_q),
//     f~ = P f~_q,   P = V Phi_q^T diag(w)   (orthonormal basis Phi).
// The result is written as [ne][3][5][nupts], the layout the volume kernels
// keep f~ in, and those kernels then take it in place of their own
// collocated flux (divergence, correction and RK update are unchanged).
#pragma once
#include "fr_kernels.cuh"

namespace frgb {

template <typename T>
struct AaOps {
  const T* BT;  // [nupts][nq]  B transposed: BT[z][q] = l_z(x_q)
  const T* PT;  // [nq][nupts]  P transposed
  int nq;
};

constexpr int kAaThreads = 128;

template <typename T, int NU>
__host__ __device__ inline bool aa_ops_staged(int nq) {
  return 2 * size_t(NU) * nq * sizeof(T) <= 64 * 1024;
}

template <typename T, int NU>
inline size_t aa_dense_smem(int nq) {
  const size_t ops = aa_ops_staged<T, NU>(nq) ? 2 * size_t(NU) * nq : 0;
  return (ops + 20 * size_t(NU) + 15 * size_t(nq)) * sizeof(T);
}

// Dense form, any element type: a persistent CTA of kAaThreads threads takes
// one element at a time.  Phase 1: one thread per quadrature point
// interpolates u (and the gradient), forms the flux and transforms it with
// the metric at that point.  Phase 2: one thread per (direction, solution
// point) projects the five variables back.  Operators live in shared memory
// when they fit (64 KB), else they are read through L1.
template <typename T, typename TR, int NU, bool NS>
__global__ void __launch_bounds__(kAaThreads)
    k_aa_flux_dense(long long ne, const T* __restrict__ uin,
                    const TR* __restrict__ X, const T* __restrict__ grad,
                    const T* __restrict__ smq, AaOps<T> gop, Phys<T> ph,
                    T* __restrict__ tf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int nq = gop.nq;
  const bool staged = aa_ops_staged<T, NU>(nq);
  const T* BT = gop.BT;
  const T* PT = gop.PT;
  T* buf = sm;
  if (staged) {
    T* b = sm;
    T* p = sm + NU * nq;
    for (int i = threadIdx.x; i < NU * nq; i += blockDim.x) {
      b[i] = gop.BT[i];
      p[i] = gop.PT[i];
    }
    BT = b;
    PT = p;
    buf = sm + 2 * NU * nq;
  }
  T* us = buf;            // [20][NU]: u, then the gradient (NS)
  T* fq = us + 20 * NU;   // [15][nq]: f~ at the quadrature points
  for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
    for (int i = threadIdx.x; i < 5 * NU; i += blockDim.x)
      us[i] = uin ? uin[e * 5 * NU + i] : T(X[e * 5 * NU + i]);
    if (NS)
      for (int i = threadIdx.x; i < 15 * NU; i += blockDim.x)
        us[5 * NU + i] = grad[e * 15 * NU + i];
    __syncthreads();
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      T uq[5] = {0, 0, 0, 0, 0};
      T gq[3][5];
      if (NS) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 5; ++k) gq[j][k] = T(0);
      }
      for (int z = 0; z < NU; ++z) {
        const T b = BT[z * nq + q];
#pragma unroll
        for (int k = 0; k < 5; ++k) uq[k] += b * us[k * NU + z];
        if (NS) {
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 5; ++k) gq[j][k] += b * us[(5 + j * 5 + k) * NU + z];
        }
      }
      T F[3][5];
      euler_flux(uq, ph, F);
      if (NS) viscous_flux_acc(uq, gq, ph, T(-1), F);
      T S[3][3];
#pragma unroll
      for (int r = 0; r < 9; ++r) S[r / 3][r % 3] = smq[(e * 9 + r) * nq + q];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k)
          fq[(d * 5 + k) * nq + q] = S[d][0] * F[0][k] + S[d][1] * F[1][k] + S[d][2] * F[2][k];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < 3 * NU; o += blockDim.x) {
      const int d = o / NU, z = o - d * NU;
      T acc[5] = {0, 0, 0, 0, 0};
      for (int q = 0; q < nq; ++q) {
        const T pw = PT[q * NU + z];
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += pw * fq[(d * 5 + k) * nq + q];
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) tf[(e * 15 + d * 5 + k) * NU + z] = acc[k];
    }
    __syncthreads();
  }
}

}  // namespace frgb
