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

// ---------------------------------------------------------------------------
// Dense form with the operators resident in shared memory and E elements per
// pass.  Solution-point and rule-point counts are padded to a multiple of
// W = 16 / sizeof(T) (zero rows / columns), so the per-element operands
// that every thread of a pass reads alike (the element's u and gradient in
// phase 1, its transformed flux at the rule points in phase 2) come as
// 16-byte broadcast loads: W FMAs per load of those operands.
template <typename T>
__host__ __device__ constexpr int aa_w() { return 16 / int(sizeof(T)); }
__host__ __device__ inline int aa_ru(int n, int w) { return (n + w - 1) / w * w; }

template <typename T, int NU>
inline size_t aa_dense_v_smem(int nq, int epb) {
  constexpr int W = aa_w<T>();
  const int nup = aa_ru(NU, W), nqp = aa_ru(nq, W);
  return (2 * size_t(nup) * nqp + size_t(epb) * (20 * nup + 15 * nqp)) * sizeof(T);
}

// 256 threads: the resident operators (up to 41 KB) are shared by more warps
constexpr int kAaVThreads = 256;

template <typename T, typename TR, int NU, bool NS>
__global__ void __launch_bounds__(kAaVThreads)
    k_aa_flux_dense_v(long long ne, int epb, const T* __restrict__ uin,
                      const TR* __restrict__ X, const T* __restrict__ grad,
                      const T* __restrict__ smq, AaOps<T> gop, Phys<T> ph,
                      T* __restrict__ tf) {
  constexpr int W = aa_w<T>();
  constexpr int NUP = (NU + W - 1) / W * W;
  using V = uint4;  // 16 bytes of W values
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nq = gop.nq, nqp = aa_ru(nq, W);
  T* BT = reinterpret_cast<T*>(smem_raw);  // [NUP][nqp]
  T* PT = BT + NUP * nqp;                   // [nqp][NUP]
  T* us = PT + NUP * nqp;                   // [epb][20][NUP]
  T* fq = us + epb * 20 * NUP;              // [epb][15][nqp]
  for (int i = threadIdx.x; i < NUP * nqp; i += blockDim.x) {
    const int z = i / nqp, q = i - z * nqp;
    BT[i] = (z < NU && q < nq) ? gop.BT[z * nq + q] : T(0);
    const int q2 = i / NUP, z2 = i - q2 * NUP;
    PT[i] = (z2 < NU && q2 < nq) ? gop.PT[q2 * NU + z2] : T(0);
  }
  for (int i = threadIdx.x; i < epb * 20 * NUP; i += blockDim.x) us[i] = T(0);
  __syncthreads();
  const int nf = NS ? 20 : 5;
  for (long long e0 = (long long)blockIdx.x * epb; e0 < ne; e0 += (long long)gridDim.x * epb) {
    const int ecnt = int(ne - e0 < epb ? ne - e0 : epb);
    for (int i = threadIdx.x; i < ecnt * 5 * NU; i += blockDim.x) {
      const int le = i / (5 * NU), r = i - le * 5 * NU, k = r / NU, z = r - k * NU;
      const long long g = (e0 + le) * 5 * NU + r;
      us[(le * 20 + k) * NUP + z] = uin ? uin[g] : T(X[g]);
    }
    if (NS)
      for (int i = threadIdx.x; i < ecnt * 15 * NU; i += blockDim.x) {
        const int le = i / (15 * NU), r = i - le * 15 * NU, c = r / NU, z = r - c * NU;
        us[(le * 20 + 5 + c) * NUP + z] = grad[(e0 + le) * 15 * NU + r];
      }
    __syncthreads();
    // phase 1: one thread per (element, rule point)
    for (int it = threadIdx.x; it < ecnt * nqp; it += blockDim.x) {
      const int le = it / nqp, q = it - le * nqp;
      const T* ue = us + le * 20 * NUP;
      T* fe = fq + le * 15 * nqp;
      if (q >= nq) {
#pragma unroll
        for (int c = 0; c < 15; ++c) fe[c * nqp + q] = T(0);
        continue;
      }
      T acc[20];
#pragma unroll
      for (int k = 0; k < 20; ++k) acc[k] = T(0);
      for (int z0 = 0; z0 < NUP; z0 += W) {
        T b[W];
#pragma unroll
        for (int w = 0; w < W; ++w) b[w] = BT[(z0 + w) * nqp + q];
#pragma unroll
        for (int k = 0; k < 20; ++k) {
          if (k >= nf) break;
          const V r = *reinterpret_cast<const V*>(ue + k * NUP + z0);
          const T* v = reinterpret_cast<const T*>(&r);
#pragma unroll
          for (int w = 0; w < W; ++w) acc[k] += b[w] * v[w];
        }
      }
      T F[3][5];
      euler_flux(acc, ph, F);
      if (NS) {
        T gq[3][5];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 5; ++k) gq[j][k] = acc[5 + j * 5 + k];
        viscous_flux_acc(acc, gq, ph, T(-1), F);
      }
      T S[3][3];
      const long long e = e0 + le;
#pragma unroll
      for (int r = 0; r < 9; ++r) S[r / 3][r % 3] = smq[(e * 9 + r) * nq + q];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k)
          fe[(d * 5 + k) * nqp + q] = S[d][0] * F[0][k] + S[d][1] * F[1][k] + S[d][2] * F[2][k];
    }
    __syncthreads();
    // phase 2: one thread per (element, direction, solution point), the
    // five variables of that direction
    for (int it = threadIdx.x; it < ecnt * 3 * NU; it += blockDim.x) {
      const int le = it / (3 * NU), r = it - le * 3 * NU, d = r / NU, z = r - d * NU;
      const T* fe = fq + (le * 15 + d * 5) * nqp;
      T acc[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) acc[c] = T(0);
      for (int q0 = 0; q0 < nqp; q0 += W) {
        T p[W];
#pragma unroll
        for (int w = 0; w < W; ++w) p[w] = PT[(q0 + w) * NUP + z];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const V rv = *reinterpret_cast<const V*>(fe + c * nqp + q0);
          const T* v = reinterpret_cast<const T*>(&rv);
#pragma unroll
          for (int w = 0; w < W; ++w) acc[c] += p[w] * v[w];
        }
      }
      const long long e = e0 + le;
#pragma unroll
      for (int c = 0; c < 5; ++c) tf[(e * 15 + d * 5 + c) * NU + z] = acc[c];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Hexahedra, sum-factorised.  The basis, the solution points and the rule are
// tensor products, so B = B1 (x) B1 (x) B1 and P = P1 (x) P1 (x) P1 with the 1D
// factors B1[i][a] = l_a(x_i) (Q rule points, N solution points per line) and
// P1[a][i] = w_i sum_m psi_m(x_a) psi_m(x_i) (orthonormal Legendre psi).
// Each operator is applied one direction at a time: 20 fields (u and the
// gradient) go N -> Q along x, y, z; the transformed flux (15 fields) comes
// back Q -> N along z, y, x.  One thread takes one line of a pass (N loads,
// Q outputs or the reverse), so shared memory is read once per line.
constexpr int kAaQMax = 13;  // qdeg <= 24

template <typename T>
struct HexAaOps {
  T b1[kAaQMax][5];  // [Q][N]
  T p1[5][kAaQMax];  // [N][Q]
  int q;
};

// Field strides of the layouts read by whole warps across field boundaries
// ([f][c][j][i] in buffer A, [f][k][j][i] in buffer B): padded to the
// smallest value >= the field's size that is congruent to Q^2 modulo 32
// banks, so a warp whose lines continue into the next field keeps distinct
// banks.
__host__ __device__ inline int hex_aa_pad(int size, int q) {
  return size + (((q * q - size) % 32) + 32) % 32;
}
__host__ __device__ inline int hex_aa_fsa(int n, int q) { return hex_aa_pad(n * q * q, q); }
__host__ __device__ inline int hex_aa_fsb(int q) { return hex_aa_pad(q * q * q, q); }
// shared memory of one element: ping-pong buffers A and B (T values)
__host__ __device__ inline int hex_aa_buf_a(int n, int q) {
  const int t = 20 * n * n * n, u = 20 * hex_aa_fsa(n, q);
  return t > u ? t : u;
}
__host__ __device__ inline int hex_aa_buf_b(int n, int q) {
  const int t = 20 * q * n * n, u = 20 * hex_aa_fsb(q);
  return t > u ? t : u;
}
constexpr int kAaOpsT = 2 * kAaQMax * 5;  // staged b1 and p1 (T values)

// One line of N values from / to global memory; 16-byte vector accesses when
// a line is a whole number of them (every line then starts 16-byte aligned).
template <int N, typename S, typename T>
__device__ __forceinline__ void aa_line_load(const S* __restrict__ p, T* v) {
  if constexpr ((N * sizeof(S)) % 16 == 0) {
    constexpr int W = 16 / sizeof(S);
#pragma unroll
    for (int j = 0; j < N / W; ++j) {
      const uint4 r = *reinterpret_cast<const uint4*>(p + j * W);
      const S* s = reinterpret_cast<const S*>(&r);
#pragma unroll
      for (int a = 0; a < W; ++a) v[j * W + a] = T(s[a]);
    }
  } else {
#pragma unroll
    for (int a = 0; a < N; ++a) v[a] = T(p[a]);
  }
}

template <int N, typename T>
__device__ __forceinline__ void aa_line_store(T* __restrict__ p, const T* v) {
  if constexpr ((N * sizeof(T)) % 16 == 0) {
    constexpr int W = 16 / sizeof(T);
#pragma unroll
    for (int j = 0; j < N / W; ++j) {
      uint4 r;
      T* s = reinterpret_cast<T*>(&r);
#pragma unroll
      for (int a = 0; a < W; ++a) s[a] = v[j * W + a];
      *reinterpret_cast<uint4*>(p + j * W) = r;
    }
  } else {
#pragma unroll
    for (int a = 0; a < N; ++a) p[a] = v[a];
  }
}
template <typename T>
inline size_t hex_aa_smem(int n, int q) {
  return size_t(kAaOpsT + hex_aa_buf_a(n, q) + hex_aa_buf_b(n, q)) * sizeof(T);
}

// QT > 0: the rule's point count per direction is a compile-time constant
// (loops unroll and the 1D coefficients are read as constant operands);
// QT = 0: any Q, coefficients from shared memory.
template <typename T, typename TR, int N, int QT, bool NS>
__global__ void __launch_bounds__(kAaThreads)
    k_hex_aa_flux(long long ne, const T* __restrict__ uin,
                  const TR* __restrict__ X, const T* __restrict__ grad,
                  const T* __restrict__ smq, HexAaOps<T> op, Phys<T> ph,
                  T* __restrict__ tf) {
  constexpr int NU = N * N * N;
  constexpr int NFLD = NS ? 20 : 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Q = QT > 0 ? QT : op.q, Q2 = Q * Q, Q3 = Q2 * Q;
  const int FA = hex_aa_fsa(N, Q), FB = hex_aa_fsb(Q);
  T* b1 = reinterpret_cast<T*>(smem_raw);  // [Q][N]
  T* p1 = b1 + kAaQMax * 5;                // [N][Q]
  T* A = b1 + kAaOpsT;
  T* Bf = A + hex_aa_buf_a(N, Q);
  const int t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < Q * N; i += nt) {
    b1[i] = op.b1[i / N][i % N];
    p1[i] = op.p1[i / Q][i % Q];
  }
  auto cb = [&](int i, int a) -> T { return QT > 0 ? op.b1[i][a] : b1[i * N + a]; };
  auto cp = [&](int a, int i) -> T { return QT > 0 ? op.p1[a][i] : p1[a * Q + i]; };
  __syncthreads();
  for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
    // x: u (5 fields), then the gradient (15), read line by line from
    // global memory: [f][c][b][a] -> Bf[f][c][b][i]
    for (int l = t; l < NFLD * N * N; l += nt) {
      T in[N];
      if (l >= 5 * N * N)
        aa_line_load<N>(grad + e * 15 * NU + (l - 5 * N * N) * N, in);
      else if (uin)
        aa_line_load<N>(uin + e * 5 * NU + l * N, in);
      else
        aa_line_load<N>(X + e * 5 * NU + l * N, in);
#pragma unroll
      for (int i = 0; i < (QT > 0 ? QT : Q); ++i) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a) s += cb(i, a) * in[a];
        Bf[l * Q + i] = s;
      }
    }
    __syncthreads();
    // y: Bf[f][c][b][i] -> A[f][c][j][i]   (line = (f, c), i)
    for (int l = t; l < NFLD * N * Q; l += nt) {
      const int fc = l / Q, i = l - fc * Q, f = fc / N, c = fc - f * N;
      T in[N];
#pragma unroll
      for (int b = 0; b < N; ++b) in[b] = Bf[(fc * N + b) * Q + i];
#pragma unroll
      for (int j = 0; j < (QT > 0 ? QT : Q); ++j) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < N; ++b) s += cb(j, b) * in[b];
        A[f * FA + (c * Q + j) * Q + i] = s;
      }
    }
    __syncthreads();
    // z: A[f][c][j][i] -> Bf[f][k][j][i]   (line = f, (j, i))
    for (int l = t; l < NFLD * Q2; l += nt) {
      const int f = l / Q2, ji = l - f * Q2;
      T in[N];
#pragma unroll
      for (int c = 0; c < N; ++c) in[c] = A[f * FA + c * Q2 + ji];
#pragma unroll
      for (int k = 0; k < (QT > 0 ? QT : Q); ++k) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < N; ++c) s += cb(k, c) * in[c];
        Bf[f * FB + k * Q2 + ji] = s;
      }
    }
    __syncthreads();
    // flux at every quadrature point, transformed, written in place
    for (int pt = t; pt < Q3; pt += nt) {
      T uq[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) uq[k] = Bf[k * FB + pt];
      T F[3][5];
      euler_flux(uq, ph, F);
      if (NS) {
        T g[3][5];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 5; ++k) g[j][k] = Bf[(5 + j * 5 + k) * FB + pt];
        viscous_flux_acc(uq, g, ph, T(-1), F);
      }
      T S[3][3];
#pragma unroll
      for (int r = 0; r < 9; ++r)
        S[r / 3][r % 3] = smq[(e * 9 + r) * Q3 + pt];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k)
          Bf[(d * 5 + k) * FB + pt] = S[d][0] * F[0][k] + S[d][1] * F[1][k] + S[d][2] * F[2][k];
    }
    __syncthreads();
    // z back: Bf[f][k][j][i] -> A[f][c][j][i]
    for (int l = t; l < 15 * Q2; l += nt) {
      const int f = l / Q2, ji = l - f * Q2;
      T acc[N];
#pragma unroll
      for (int c = 0; c < N; ++c) acc[c] = T(0);
#pragma unroll
      for (int k = 0; k < (QT > 0 ? QT : Q); ++k) {
        const T v = Bf[f * FB + k * Q2 + ji];
#pragma unroll
        for (int c = 0; c < N; ++c) acc[c] += cp(c, k) * v;
      }
#pragma unroll
      for (int c = 0; c < N; ++c) A[f * FA + c * Q2 + ji] = acc[c];
    }
    __syncthreads();
    // y back: A[f][c][j][i] -> Bf[f][c][b][i]
    for (int l = t; l < 15 * N * Q; l += nt) {
      const int fc = l / Q, i = l - fc * Q, f = fc / N, c = fc - f * N;
      T acc[N];
#pragma unroll
      for (int b = 0; b < N; ++b) acc[b] = T(0);
#pragma unroll
      for (int j = 0; j < (QT > 0 ? QT : Q); ++j) {
        const T v = A[f * FA + (c * Q + j) * Q + i];
#pragma unroll
        for (int b = 0; b < N; ++b) acc[b] += cp(b, j) * v;
      }
#pragma unroll
      for (int b = 0; b < N; ++b) Bf[(fc * N + b) * Q + i] = acc[b];
    }
    __syncthreads();
    // x back: Bf[f][c][b][i] -> tf[e][f][c][b][a]
    for (int l = t; l < 15 * N * N; l += nt) {
      T acc[N];
#pragma unroll
      for (int a = 0; a < N; ++a) acc[a] = T(0);
#pragma unroll
      for (int i = 0; i < (QT > 0 ? QT : Q); ++i) {
        const T v = Bf[l * Q + i];
#pragma unroll
        for (int a = 0; a < N; ++a) acc[a] += cp(a, i) * v;
      }
      aa_line_store<N>(tf + e * 15 * NU + l * N, acc);
    }
    __syncthreads();
  }
}

}  // namespace frgb
