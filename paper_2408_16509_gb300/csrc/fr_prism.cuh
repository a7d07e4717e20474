// Prism kernels that use the structure of the prism's operators (Section 3.1,
// "Matrix multiplications": the operator matrices are sparse, and kernels
// that skip their zeros do less work than dense products).
//
// The prism's solution points are the triangle points times the line
// points (point z * NT + t: triangle point t on line level z) and its basis
// is the triangle basis times the line basis, so
//   D_xi, D_eta   act within a level: sum_t' A_xi[t][t'] u(t', z)
//   D_zeta        acts along a line:  sum_z' B[z][z'] u(t, z')
// and the interpolation to a flux point (M0) and the correction lift (LIFT)
// touch few points (the line through a triangle-face point, the edge
// points of a level for a quadrilateral face).  The host reads A_xi, A_eta,
// B and the nonzeros of M0 and LIFT out of the element's dense operators
// and checks the structure (`build_prism_ops`); the kernels below then do
// what k_grad_dense / k_vol_dense do with those operators: per solution
// point 2 NT + NL line terms instead of 3 NU dense ones for the
// derivatives, and a handful of terms per row of M0 and LIFT.
#pragma once
#include <cstdint>

#include "fr_kernels.cuh"

namespace frgb {

template <typename T>
struct PriOps {
  const T* Axi;    // [NT][NT]  D_xi within a level
  const T* Aeta;   // [NT][NT]  D_eta within a level
  const T* B;      // [NL][NL]  D_zeta along a line
  const int* Mc;   // [NF][nm]  nonzero columns of M0 (solution points)
  const T* Mv;     // [NF][nm]  their values (0 past a row's count)
  const int* Lc;   // [NU][nl]  nonzero columns of LIFT (flux points)
  const T* Lv;     // [NU][nl]
  const T* NREF;   // [NF][3]   reference normals
  int nm, nl;      // entries per row (rows shorter than that are padded)
};

// prism order of (NU, NF): NT = (p+1)(p+2)/2, NL = p+1, NU = NT NL,
// NF = 2 NT + 3 NL^2; 0 if (NU, NF) is no prism
__host__ __device__ constexpr int pri_order(int nu, int nf) {
  for (int p = 1; p <= 8; ++p) {
    const int nt = (p + 1) * (p + 2) / 2, nl = p + 1;
    if (nu == nt * nl && nf == 2 * nt + 3 * nl * nl) return p;
  }
  return 0;
}

// Shared-memory image of PriOps: T arrays first (A_xi, A_eta, B, Mv, Lv,
// NREF), then the int arrays (Mc, Lc).
template <typename T, int NU, int NF>
struct PriLayout {
  static constexpr int P = pri_order(NU, NF);
  static constexpr int NT = (P + 1) * (P + 2) / 2, NL = P + 1;
  __host__ __device__ static constexpr int tcount(int nm, int nl) {
    return 2 * NT * NT + NL * NL + NF * nm + NU * nl + 3 * NF;
  }
  // the staged operators, 16-byte padded (the element arrays follow)
  __host__ __device__ static constexpr int bytes(int nm, int nl) {
    return ((tcount(nm, nl) * int(sizeof(T)) + 15) / 16 * 16) +
           ((NF * nm + NU * nl) * 4 + 15) / 16 * 16;
  }
};

// the upper bounds the kernels are built for (entries per row of M0 and
// LIFT); the host falls back to the dense kernels above them
constexpr int kPriMaxM0 = 16, kPriMaxLift = 64;

template <typename T, int NU, int NF>
__device__ __forceinline__ PriOps<T> stage_pri_ops(const PriOps<T>& g, unsigned char* raw) {
  using PL = PriLayout<T, NU, NF>;
  constexpr int NT = PL::NT, NL = PL::NL;
  T* s = reinterpret_cast<T*>(raw);
  T* axi = s;
  T* aeta = axi + NT * NT;
  T* b = aeta + NT * NT;
  T* mv = b + NL * NL;
  T* lv = mv + NF * g.nm;
  T* nr = lv + NU * g.nl;
  int* mc = reinterpret_cast<int*>(raw + ((PL::tcount(g.nm, g.nl) * int(sizeof(T)) + 15) / 16 * 16));
  int* lc = mc + NF * g.nm;
  for (int i = threadIdx.x; i < NT * NT; i += blockDim.x) {
    axi[i] = g.Axi[i];
    aeta[i] = g.Aeta[i];
  }
  for (int i = threadIdx.x; i < NL * NL; i += blockDim.x) b[i] = g.B[i];
  for (int i = threadIdx.x; i < NF * g.nm; i += blockDim.x) {
    mv[i] = g.Mv[i];
    mc[i] = g.Mc[i];
  }
  for (int i = threadIdx.x; i < NU * g.nl; i += blockDim.x) {
    lv[i] = g.Lv[i];
    lc[i] = g.Lc[i];
  }
  for (int i = threadIdx.x; i < 3 * NF; i += blockDim.x) nr[i] = g.NREF[i];
  __syncthreads();
  return PriOps<T>{axi, aeta, b, mc, mv, lc, lv, nr, g.nm, g.nl};
}

// NS gradient path on prisms (as k_grad_dense): corrected reference
// gradient, physical gradient at the solution points (global and shared),
// its values at the flux points (q form: the viscous normal flux there).
template <typename T, int NU, int NF, int EPB, bool QV>
__global__ void __launch_bounds__(EPB* NU)
    k_grad_pri(long long ne, const T* __restrict__ u, const T* __restrict__ du,
               const T* __restrict__ smat, const T* __restrict__ rcpdjac, PriOps<T> gops,
               T* __restrict__ grad, ViscArgs<T> va, BCTab<T> bc, Phys<T> ph) {
  using L = DenseLayout<T, NU, NF>;
  using PL = PriLayout<T, NU, NF>;
  constexpr int NT = PL::NT, NL = PL::NL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PriOps<T> op = stage_pri_ops<T, NU, NF>(gops, smem_raw);
  T* buf = reinterpret_cast<T*>(smem_raw + PL::bytes(gops.nm, gops.nl));
  const int le = threadIdx.x / NU, z = threadIdx.x % NU;
  const int lz = z / NT, lt = z - lz * NT;  // level and triangle point
  T* us = buf + le * L::kGradElem;
  T* ds = us + (L::kRows ? L::kP5 * NU : 5 * NU);
  T* gs = ds + (L::kRows ? L::kP5 * NF : 5 * NF);
  const long long ngroups = (ne + EPB - 1) / EPB;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long long e = grp * EPB + le;
    const bool act = e < ne;
    if (act) {
      T v[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = u[(e * 5 + k) * NU + z];
      put5<L, NU>(us, z, v);
      for (int f = z; f < NF; f += NU) {
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = du[(e * 5 + k) * NF + f];
        put5<L, NF>(ds, f, v);
      }
    }
    __syncthreads();
    if (act) {
      T gref[3][5];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k) gref[d][k] = T(0);
      // xi, eta: the points of this level (the same rows for every thread of
      // the level: broadcast reads)
#pragma unroll 2
      for (int t2 = 0; t2 < NT; ++t2) {
        T v[5];
        get5<L, NU>(us, lz * NT + t2, v);
        const T ax = op.Axi[lt * NT + t2], ay = op.Aeta[lt * NT + t2];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          gref[0][k] += ax * v[k];
          gref[1][k] += ay * v[k];
        }
      }
      // zeta: the points of this line
#pragma unroll
      for (int z2 = 0; z2 < NL; ++z2) {
        T v[5];
        get5<L, NU>(us, z2 * NT + lt, v);
        const T bz = op.B[lz * NL + z2];
#pragma unroll
        for (int k = 0; k < 5; ++k) gref[2][k] += bz * v[k];
      }
      // correction: LIFT (n~ du), the few flux points that reach this point
      for (int j = 0; j < op.nl; ++j) {
        const int f = op.Lc[z * op.nl + j];
        const T l = op.Lv[z * op.nl + j];
        T dq[5];
        get5<L, NF>(ds, f, dq);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T w = l * op.NREF[f * 3 + d];
#pragma unroll
          for (int k = 0; k < 5; ++k) gref[d][k] += w * dq[k];
        }
      }
      T S[3][3];
#pragma unroll
      for (int r = 0; r < 9; ++r) S[r / 3][r % 3] = smat[(e * 9 + r) * NU + z];
      const T rj = rcpdjac[e * NU + z];
      T gg[15];
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          gg[j * 5 + k] = rj * (S[0][j] * gref[0][k] + S[1][j] * gref[1][k] +
                                S[2][j] * gref[2][k]);
          grad[(e * 15 + j * 5 + k) * NU + z] = gg[j * 5 + k];
        }
      put15<L, NU>(gs, z, gg);
    }
    __syncthreads();
    if (act) {
      for (int f = z; f < NF; f += NU) {
        T acc[15];
#pragma unroll
        for (int c = 0; c < 15; ++c) acc[c] = T(0);
        for (int j = 0; j < op.nm; ++j) {
          const int q = op.Mc[f * op.nm + j];
          const T m = op.Mv[f * op.nm + j];
          T g[15];
          get15<L, NU>(gs, q, g);
#pragma unroll
          for (int c = 0; c < 15; ++c) acc[c] += m * g[c];
        }
        if (QV) {
          write_visc_q(va, bc, ph, e, f, NF, acc);
        } else {
#pragma unroll
          for (int c = 0; c < 15; ++c) va.q[(e * 15 + c) * NF + f] = acc[c];
        }
      }
    }
    __syncthreads();
  }
}

// Volume kernel on prisms (as k_vol_dense): f~ = S F at the solution points,
// Eq. (FRfinal) div = sum_d D_d f~_d + LIFT (F^C - n~.M0 f~), R = -div/J,
// the RK epilogue and the next stage's u_f = M0 u_next.
template <typename T, int NU, int NF, int EPB, bool NS>
__global__ void __launch_bounds__(EPB* NU)
    k_vol_pri(long long ne, const T* __restrict__ u, const T* __restrict__ grad,
              const T* __restrict__ fc, const T* __restrict__ smat,
              const T* __restrict__ rcpdjac, PriOps<T> gops, Phys<T> ph, StageArgs<T> sa) {
  using L = DenseLayout<T, NU, NF>;
  using PL = PriLayout<T, NU, NF>;
  constexpr int NT = PL::NT, NL = PL::NL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PriOps<T> op = stage_pri_ops<T, NU, NF>(gops, smem_raw);
  T* buf = reinterpret_cast<T*>(smem_raw + PL::bytes(gops.nm, gops.nl));
  const int le = threadIdx.x / NU, z = threadIdx.x % NU;
  const int lz = z / NT, lt = z - lz * NT;
  T* ft = buf + le * L::kVolElem;  // f~ (component d * 5 + k), then u_next
  T* jm = ft + (L::kRows ? 16 * NU : 15 * NU);
  const long long ngroups = (ne + EPB - 1) / EPB;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long long e = grp * EPB + le;
    const bool act = e < ne;
    T uz[5];
    if (act) {
#pragma unroll
      for (int k = 0; k < 5; ++k) uz[k] = u[(e * 5 + k) * NU + z];
      T F[3][5];
      euler_flux(uz, ph, F);
      if (NS) {
        T g[3][5];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int k = 0; k < 5; ++k) g[j][k] = grad[(e * 15 + j * 5 + k) * NU + z];
        viscous_flux_acc(uz, g, ph, T(-1), F);
      }
      T S[3][3];
#pragma unroll
      for (int r = 0; r < 9; ++r) S[r / 3][r % 3] = smat[(e * 9 + r) * NU + z];
      T fv[15];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 5; ++k)
          fv[d * 5 + k] = S[d][0] * F[0][k] + S[d][1] * F[1][k] + S[d][2] * F[2][k];
      put15<L, NU>(ft, z, fv);
    }
    __syncthreads();
    if (act) {
      // jump at every flux point: F^C - n~ . M0 f~
      for (int f = z; f < NF; f += NU) {
        const T n0 = op.NREF[f * 3], n1 = op.NREF[f * 3 + 1], n2 = op.NREF[f * 3 + 2];
        T fn[5] = {0, 0, 0, 0, 0};
        for (int j = 0; j < op.nm; ++j) {
          const int q = op.Mc[f * op.nm + j];
          const T m = op.Mv[f * op.nm + j];
          T v[15];
          get15<L, NU>(ft, q, v);
          const T w0 = m * n0, w1 = m * n1, w2 = m * n2;
#pragma unroll
          for (int k = 0; k < 5; ++k) fn[k] += w0 * v[k] + w1 * v[5 + k] + w2 * v[10 + k];
        }
        T jv[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) jv[k] = fc[(e * 5 + k) * NF + f] - fn[k];
        put5<L, NF>(jm, f, jv);
      }
    }
    __syncthreads();
    T s[5];
    if (act) {
      T div[5] = {0, 0, 0, 0, 0};
#pragma unroll 2
      for (int t2 = 0; t2 < NT; ++t2) {
        T v[15];
        get15<L, NU>(ft, lz * NT + t2, v);
        const T ax = op.Axi[lt * NT + t2], ay = op.Aeta[lt * NT + t2];
#pragma unroll
        for (int k = 0; k < 5; ++k) div[k] += ax * v[k] + ay * v[5 + k];
      }
#pragma unroll
      for (int z2 = 0; z2 < NL; ++z2) {
        T v[15];
        get15<L, NU>(ft, z2 * NT + lt, v);
        const T bz = op.B[lz * NL + z2];
#pragma unroll
        for (int k = 0; k < 5; ++k) div[k] += bz * v[10 + k];
      }
      for (int j = 0; j < op.nl; ++j) {
        const int f = op.Lc[z * op.nl + j];
        const T l = op.Lv[z * op.nl + j];
        T jv[5];
        get5<L, NF>(jm, f, jv);
#pragma unroll
        for (int k = 0; k < 5; ++k) div[k] += l * jv[k];
      }
      const T rj = rcpdjac[e * NU + z];
      T R[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) R[k] = -div[k] * rj;
      stage_update(sa, e * 5 * NU + z, NU, uz, R, s);
    }
    if (sa.uf_next != nullptr) {
      __syncthreads();  // ft no longer read: reuse it for the next stage value
      if (act) put5<L, NU>(ft, z, s);
      __syncthreads();
      if (act) {
        for (int f = z; f < NF; f += NU) {
          T acc[5] = {0, 0, 0, 0, 0};
          for (int j = 0; j < op.nm; ++j) {
            const int q = op.Mc[f * op.nm + j];
            const T m = op.Mv[f * op.nm + j];
            T v[5];
            get5<L, NU>(ft, q, v);
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[k] += m * v[k];
          }
#pragma unroll
          for (int k = 0; k < 5; ++k) sa.uf_next[(e * 5 + k) * NF + f] = acc[k];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace frgb
