// FR right-hand-side kernels (PyFR v2.0.3, Section 2) -- generic dense form.
//
// Device layouts, per element type, element-major with the variable index
// between the element and the point index so that one warp reads 32
// consecutive points of one variable:
//   solution / stage registers   [ne][5][nupts]
//   flux-point traces            [ne][5][nfpts]   (one buffer for all types)
//   gradients at solution pts    [ne][3*5][nupts]
//   gradients at flux pts        [ne][3*5][nfpts]
//   metric S = det J J^{-1}      [ne][9][nupts]  and 1/det J [ne][nupts]
// Operators are stored transposed so that consecutive threads read
// consecutive entries: M0T[nupts][nfpts], DT[3][nupts][nupts] (DT[d][v][z] =
// d l_v/dx~_d at x_z), LIFTT[nfpts][nupts].
#pragma once
#include <cstdint>

#include "fr_convert.cuh"
#include "fr_phys.cuh"

namespace frgb {

constexpr int kMaxBC = 8;

// Per-type regions of the shared flux-point buffers.
struct TypeTab {
  int nf[3];
  long long off_f[3];  // offset of the type's [ne][5][nf] region
};

template <typename T>
struct BCTab {
  int kind[kMaxBC];      // 0 = given state, 1 = extrapolate, 2 = exchange
                         // (outside state of a partner part), 3 = state
                         // prescribed per boundary point (in xu)
  T state[kMaxBC][5];    // conserved ghost state
};

template <typename T>
struct DenseOps {
  const T* M0T;    // [nu][nf]
  const T* DT;     // [3][nu][nu]
  const T* LIFTT;  // [nf][nu]
  const T* NREF;   // [nf][3]
  // M0 by its nonzeros ([nf][nm] columns and values), nm = 0: dense M0.
  // Tetrahedra: every flux point is a solution point (nm = 1, a gather).
  const int* Mc = nullptr;
  const T* Mv = nullptr;
  int nm = 0;
};

// Time-integration epilogue of the volume kernel.
//   mode 0: write R to out
//   mode 1: classical RK4 stage `stage`  (registers X, A, Y)
//   mode 2: RK4(3)5[2R+] stage `stage`   (registers X, Y)
template <typename T>
struct StageArgs {
  int mode, stage;
  T* X;
  T* A;
  T* Y;
  T* out;
  const double* dt;  // device scalar
  int* flag;         // non-finite flag (bit 0)
  T* uf_next;        // flux-point buffer for the next stage (or nullptr)
  T* E = nullptr;    // embedded-error register of an adaptive step (or nullptr)
};

// RK4(3)5[2R+]C of Kennedy, Carpenter & Lewis (2000): the sub-diagonal
// a_{i+1,i} of the two-register scheme, the weights b and b - bhat with the
// embedded third-order weights bhat of the same publication.  Statically
// initialised: every translation unit holds its own copy.
static __constant__ double c_rk45_a[4] = {
    970286171893.0 / 4311952581923.0, 6584761158862.0 / 12103376702013.0,
    2251764453980.0 / 15575788980749.0, 26877169314380.0 / 34165994151039.0};
static __constant__ double c_rk45_b[5] = {
    1153189308089.0 / 22510343858157.0, 1772645290293.0 / 4653164025191.0,
    -1672844663538.0 / 4480602732383.0, 2114624349019.0 / 3568978502595.0,
    5198255086312.0 / 14908931495163.0};
static __constant__ double c_rk45_e[5] = {
    1153189308089.0 / 22510343858157.0 - 1016888040809.0 / 7410784769900.0,
    1772645290293.0 / 4653164025191.0 - 11231460423587.0 / 58533540763752.0,
    -1672844663538.0 / 4480602732383.0 + 1563879915014.0 / 6823010717585.0,
    2114624349019.0 / 3568978502595.0 - 606302364029.0 / 971179775848.0,
    5198255086312.0 / 14908931495163.0 - 1097981568119.0 / 3980877426909.0};

// The same coefficients rounded once to FP32, for the mixed form's FP32
// increments (b dt r and friends are formed in FP32 there).
static __constant__ float c_rk45_af[4] = {
    float(970286171893.0 / 4311952581923.0), float(6584761158862.0 / 12103376702013.0),
    float(2251764453980.0 / 15575788980749.0), float(26877169314380.0 / 34165994151039.0)};
static __constant__ float c_rk45_bf[5] = {
    float(1153189308089.0 / 22510343858157.0), float(1772645290293.0 / 4653164025191.0),
    float(-1672844663538.0 / 4480602732383.0), float(2114624349019.0 / 3568978502595.0),
    float(5198255086312.0 / 14908931495163.0)};
static __constant__ float c_rk45_ef[5] = {
    float(1153189308089.0 / 22510343858157.0 - 1016888040809.0 / 7410784769900.0),
    float(1772645290293.0 / 4653164025191.0 - 11231460423587.0 / 58533540763752.0),
    float(-1672844663538.0 / 4480602732383.0 + 1563879915014.0 / 6823010717585.0),
    float(2114624349019.0 / 3568978502595.0 - 606302364029.0 / 971179775848.0),
    float(5198255086312.0 / 14908931495163.0 - 1097981568119.0 / 3980877426909.0)};

__device__ __forceinline__ void decode_fp(int32_t code, const TypeTab& tt,
                                          int* t, long long* e, int* f) {
  *t = code >> 29;
  long long local = code & ((1 << 29) - 1);
  int nf = tt.nf[*t];
  *e = local / (5 * nf);
  *f = int(local - *e * 5 * nf);
}

// index of variable v, point f, element e in a [ne][nv][nf] region of type t
__device__ __forceinline__ long long fp_index(const TypeTab& tt, int t,
                                              long long e, int f, int nv,
                                              int v) {
  long long base = tt.off_f[t] / 5 * nv;  // region scales with the var count
  return base + (e * nv + v) * tt.nf[t] + f;
}

// RK epilogue for one point: R[5] -> registers; returns the next stage value
template <typename T>
__device__ __forceinline__ void stage_update(const StageArgs<T>& a,
                                             long long idx0, long long vstr,
                                             const T u[5], T R[5], T s[5]) {
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 5; ++k) bad |= !isfinite(R[k]);
  if (bad) atomicOr(a.flag, 1);
  if (a.mode == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      a.out[idx0 + k * vstr] = R[k];
      s[k] = u[k];
    }
    return;
  }
  const T dt = T(*a.dt);
  if (a.mode == 1) {
    const int st = a.stage;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      long long i = idx0 + k * vstr;
      if (st == 0) {
        T x = u[k];
        a.A[i] = x + dt * T(1.0 / 6.0) * R[k];
        s[k] = x + dt * T(0.5) * R[k];
        a.Y[i] = s[k];
      } else if (st < 3) {
        T x = a.X[i];
        a.A[i] = a.A[i] + dt * T(1.0 / 3.0) * R[k];
        s[k] = x + (st == 1 ? dt * T(0.5) : dt) * R[k];
        a.Y[i] = s[k];
      } else {
        s[k] = a.A[i] + dt * T(1.0 / 6.0) * R[k];
        a.X[i] = s[k];
      }
    }
    return;
  }
  // mode 2: two-register RK4(3)5[2R+]
  const int st = a.stage;
  const T b = T(c_rk45_b[st]);
  const T am = st < 4 ? T(c_rk45_a[st]) - b : T(0);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    long long i = idx0 + k * vstr;
    T x = (st == 0 ? u[k] : a.X[i]) + b * dt * R[k];
    a.X[i] = x;
    if (a.E) {  // error estimate dt sum_i (b_i - bhat_i) R_i
      const T ev = T(c_rk45_e[st]) * dt * R[k];
      a.E[i] = st == 0 ? ev : a.E[i] + ev;
    }
    if (st < 4) {
      s[k] = x + am * dt * R[k];
      a.Y[i] = s[k];
    } else {
      s[k] = x;
    }
  }
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copy (cp.async) of `bytes` (a multiple of 4)
// by the `nthr` threads numbered t: 16-byte chunks when both addresses and
// the size are 16-byte aligned, else 4-byte chunks.  Completes at
// cp_async_wait_all() of each issuing thread.
__device__ __forceinline__ void async_copy(void* sdst, const void* gsrc, int bytes,
                                           int t, int nthr) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(sdst));
  const unsigned long long g = reinterpret_cast<unsigned long long>(gsrc);
  if (((s | uint32_t(g) | uint32_t(bytes)) & 15u) == 0) {
    for (int i = 16 * t; i < bytes; i += 16 * nthr)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s + i), "l"(g + i)
                   : "memory");
  } else {
    for (int i = 4 * t; i < bytes; i += 4 * nthr)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s + i), "l"(g + i)
                   : "memory");
  }
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Eq. (disu): u_f = M0 u, one element per EPB group of threads.
template <typename T, int NU, int NF, int EPB>
__global__ void __launch_bounds__(EPB* NU)
    k_interp_dense(long long ne, const T* __restrict__ u, DenseOps<T> ops,
                   T* __restrict__ uf) {
  __shared__ T us[EPB][5][NU];
  const int le = threadIdx.x / NU, z = threadIdx.x % NU;
  const long long e = (long long)blockIdx.x * EPB + le;
  if (e < ne) {
#pragma unroll
    for (int k = 0; k < 5; ++k) us[le][k][z] = u[(e * 5 + k) * NU + z];
  }
  __syncthreads();
  if (e >= ne) return;
  for (int f = z; f < NF; f += NU) {
    T acc[5] = {0, 0, 0, 0, 0};
    for (int q = 0; q < NU; ++q) {
      T m = ops.M0T[q * NF + f];
#pragma unroll
      for (int k = 0; k < 5; ++k) acc[k] += m * us[le][k][q];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) uf[(e * 5 + k) * NF + f] = acc[k];
  }
}

// ---------------------------------------------------------------------------
// Eq. (comm_flux) on interior pairs: transformed common normal flux written
// to both sides (|S^T n~| F on L, -|S^T n~| F on R).  NS subtracts the BR1
// average of both sides' viscous normal fluxes.
template <typename T, bool NS>
__global__ void k_face_flux(int np, const int32_t* __restrict__ pl,
                            const int32_t* __restrict__ pr,
                            const T* __restrict__ pn, const T* __restrict__ pmr,
                            const T* __restrict__ uf, const T* __restrict__ gf,
                            T* __restrict__ fc, TypeTab tt, Phys<T> ph) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  int tl, tr, fl, frr;
  long long el, er;
  decode_fp(pl[i], tt, &tl, &el, &fl);
  decode_fp(pr[i], tt, &tr, &er, &frr);
  T ul[5], ur[5], n[3];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    ul[k] = uf[fp_index(tt, tl, el, fl, 5, k)];
    ur[k] = uf[fp_index(tt, tr, er, frr, 5, k)];
  }
  n[0] = pn[4 * i];
  n[1] = pn[4 * i + 1];
  n[2] = pn[4 * i + 2];
  T ml = pn[4 * i + 3], mr = pmr[i];
  T F[5];
  rusanov(ul, ur, n, ph, F);
  if (NS) {
    T gl[3][5], gr[3][5];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        gl[j][k] = gf[fp_index(tt, tl, el, fl, 15, j * 5 + k)];
        gr[j][k] = gf[fp_index(tt, tr, er, frr, 15, j * 5 + k)];
      }
    viscous_normal_acc(ul, gl, n, ph, -(T(0.5) + ph.beta), F);
    viscous_normal_acc(ur, gr, n, ph, -(T(0.5) - ph.beta), F);
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] += ph.tau * (ul[k] - ur[k]);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    fc[fp_index(tt, tl, el, fl, 5, k)] = ml * F[k];
    fc[fp_index(tt, tr, er, frr, 5, k)] = -mr * F[k];
  }
}

template <typename T>
__device__ __forceinline__ void ghost_state(const BCTab<T>& bc, int b,
                                            const T ul[5], T ur[5]) {
  if (bc.kind[b] == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) ur[k] = bc.state[b][k];
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k) ur[k] = ul[k];
  }
}

// Outside state of boundary point i: the condition's, or for an exchange
// point the partner part's trace and for a prescribed point the caller's
// state, both in xu ([nb][5]).
template <typename T>
__device__ __forceinline__ void ghost_state_x(const BCTab<T>& bc, int b, int i,
                                              const T* __restrict__ xu,
                                              const T ul[5], T ur[5]) {
  if (bc.kind[b] == 2 || bc.kind[b] == 3) {
#pragma unroll
    for (int k = 0; k < 5; ++k) ur[k] = xu[5 * i + k];
  } else {
    ghost_state(bc, b, ul, ur);
  }
}

// Boundary flux points: outside state from the boundary condition, outside
// gradient equal to the inside one; at exchange points both come from the
// partner part (xu [nb][5], xg [nb][15]), which makes them interior faces.
template <typename T, bool NS>
__global__ void k_bnd_flux(int nb, const int32_t* __restrict__ bidx,
                           const int32_t* __restrict__ bbc,
                           const T* __restrict__ bn, const T* __restrict__ uf,
                           const T* __restrict__ gf, T* __restrict__ fc,
                           TypeTab tt, Phys<T> ph, BCTab<T> bc,
                           const T* __restrict__ xu = nullptr,
                           const T* __restrict__ xg = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int t, f;
  long long e;
  decode_fp(bidx[i], tt, &t, &e, &f);
  T ul[5], ur[5], n[3] = {bn[4 * i], bn[4 * i + 1], bn[4 * i + 2]};
#pragma unroll
  for (int k = 0; k < 5; ++k) ul[k] = uf[fp_index(tt, t, e, f, 5, k)];
  const int b = bbc[i];
  ghost_state_x(bc, b, i, xu, ul, ur);
  T F[5];
  rusanov(ul, ur, n, ph, F);
  if (NS) {
    T g[3][5], gr[3][5];
    const bool x = bc.kind[b] == 2;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        g[j][k] = gf[fp_index(tt, t, e, f, 15, j * 5 + k)];
        gr[j][k] = x ? xg[15 * i + j * 5 + k] : g[j][k];
      }
    const T vb = x ? T(0) : ph.beta;  // exchange points: BR1 weights
    viscous_normal_acc(ul, g, n, ph, -(T(0.5) + vb), F);
    viscous_normal_acc(ur, gr, n, ph, -(T(0.5) - vb), F);
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] += ph.tau * (ul[k] - ur[k]);
  }
  T m = bn[4 * i + 3];
#pragma unroll
  for (int k = 0; k < 5; ++k) fc[fp_index(tt, t, e, f, 5, k)] = m * F[k];
}

// NS: common solution u^C = (u- + u+)/2; stores u^C - u_f on both sides.
// (LDG: u^C = (1/2 - beta) u_L + (1/2 + beta) u_R along the orientation.)
template <typename T>
__global__ void k_face_ucommon(int np, const int32_t* __restrict__ pl,
                               const int32_t* __restrict__ pr,
                               const T* __restrict__ uf, T* __restrict__ du,
                               TypeTab tt, T beta = T(0)) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  int tl, tr, fl, frr;
  long long el, er;
  decode_fp(pl[i], tt, &tl, &el, &fl);
  decode_fp(pr[i], tt, &tr, &er, &frr);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    long long il = fp_index(tt, tl, el, fl, 5, k);
    long long ir = fp_index(tt, tr, er, frr, 5, k);
    T a = uf[il], b = uf[ir];
    du[il] = (T(0.5) + beta) * (b - a);
    du[ir] = -(T(0.5) - beta) * (b - a);
  }
}

template <typename T>
__global__ void k_bnd_ucommon(int nb, const int32_t* __restrict__ bidx,
                              const int32_t* __restrict__ bbc,
                              const T* __restrict__ uf, T* __restrict__ du,
                              TypeTab tt, BCTab<T> bc,
                              const T* __restrict__ xu = nullptr, T ph_beta = T(0)) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int t, f;
  long long e;
  decode_fp(bidx[i], tt, &t, &e, &f);
  T ul[5], ur[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) ul[k] = uf[fp_index(tt, t, e, f, 5, k)];
  const int b = bbc[i];
  ghost_state_x(bc, b, i, xu, ul, ur);
  const T w = bc.kind[b] == 2 ? T(0.5) : T(0.5) + ph_beta;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    du[fp_index(tt, t, e, f, 5, k)] = w * (ur[k] - ul[k]);
}

// ---------------------------------------------------------------------------
// Viscous coupling at flux points.  Each element evaluates, at its own flux
// points, the transformed normal viscous flux q = F_v(u_f, grad u_f) .
// (S^T n~) with its own metric (S^T n~ = |S^T n~| n, Nanson); at boundary
// points q is the average over the inside state and the boundary's outside
// state, which shares the inside gradient.  The interface kernel then forms
// the BR1 average from q of both sides, so the 15 gradient components never
// leave the element.
template <typename T>
struct ViscArgs {
  const T* uf;          // this type's [ne][5][nf] solution traces
  const T* fnv;         // this type's [ne][3][nf] S^T n~ at flux points
  const int8_t* fbc;    // this type's [ne][nf]: -1 interior, else bc index
  T* q;                 // this type's [ne][5][nf] output
  const int32_t* fbi = nullptr;  // [ne][nf] boundary-point index (prescribed states)
  const T* xp = nullptr;         // [nb][5] per-point outside states
};

// Outside state of a prescribed boundary point seen from the element side
// (flux point f of element e), or nullptr.
template <typename T>
__device__ __forceinline__ const T* prescribed_at(const ViscArgs<T>& va, long long e,
                                                  int f, int nf) {
  if (!va.fbi) return nullptr;
  const int32_t i = va.fbi[e * nf + f];
  return i >= 0 ? va.xp + 5 * (long long)i : nullptr;
}

template <typename T>
__device__ __forceinline__ void write_visc_q(const ViscArgs<T>& va,
                                             const BCTab<T>& bc,
                                             const Phys<T>& ph, long long e,
                                             int f, int nf, const T g[15]) {
  T u[5], G[3][5], nv[3];
#pragma unroll
  for (int k = 0; k < 5; ++k) u[k] = va.uf[(e * 5 + k) * nf + f];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    nv[j] = va.fnv[(e * 3 + j) * nf + f];
#pragma unroll
    for (int k = 0; k < 5; ++k) G[j][k] = g[j * 5 + k];
  }
  T q[5] = {0, 0, 0, 0, 0};
  viscous_normal_acc(u, G, nv, ph, T(1), q);
  const int b = va.fbc[e * nf + f];
  if (b >= 0 && bc.kind[b] != 2) {  // exchange points keep the inside q
    T ur[5], q2[5] = {0, 0, 0, 0, 0};
    const T* pre = prescribed_at(va, e, f, nf);
    if (bc.kind[b] == 3 && pre) {
#pragma unroll
      for (int k = 0; k < 5; ++k) ur[k] = pre[k];
    } else if (bc.kind[b] == 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k) ur[k] = bc.state[b][k];
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k) ur[k] = u[k];
    }
    viscous_normal_acc(ur, G, nv, ph, T(1), q2);
#pragma unroll
    for (int k = 0; k < 5; ++k)
      q[k] = (T(0.5) + ph.beta) * q[k] + (T(0.5) - ph.beta) * q2[k];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) va.q[(e * 5 + k) * nf + f] = q[k];
}

// Viscous normal flux q of write_visc_q from inputs read beforehand: u
// (trace), G (gradient at the flux point), nv = S^T n~, b = boundary-
// condition index or -1.
template <typename T>
__device__ __forceinline__ void visc_q_pre(const BCTab<T>& bc, const Phys<T>& ph,
                                           const T u[5], const T G[3][5],
                                           const T nv[3], int b, T q[5],
                                           const T* pre = nullptr) {
#pragma unroll
  for (int k = 0; k < 5; ++k) q[k] = T(0);
  viscous_normal_acc(u, G, nv, ph, T(1), q);
  if (b >= 0 && bc.kind[b] != 2) {  // exchange points keep the inside q
    T ur[5], q2[5] = {0, 0, 0, 0, 0};
    if (bc.kind[b] == 3 && pre) {
#pragma unroll
      for (int k = 0; k < 5; ++k) ur[k] = pre[k];
    } else if (bc.kind[b] == 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k) ur[k] = bc.state[b][k];
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k) ur[k] = u[k];
    }
    viscous_normal_acc(ur, G, nv, ph, T(1), q2);
#pragma unroll
    for (int k = 0; k < 5; ++k)
      q[k] = (T(0.5) + ph.beta) * q[k] + (T(0.5) - ph.beta) * q2[k];
  }
}

// Common flux on interior pairs from the sides' viscous fluxes q:
// F^C_L = |S^T n~|_L Rus - (q_L - (m_L/m_R) q_R)/2,
// F^C_R = -|S^T n~|_R Rus + ((m_R/m_L) q_L - q_R)/2.
template <typename T>
__global__ void k_face_flux_ns(int np, const int32_t* __restrict__ pl,
                               const int32_t* __restrict__ pr,
                               const T* __restrict__ pn,
                               const T* __restrict__ pmr,
                               const T* __restrict__ uf,
                               const T* __restrict__ q, T* __restrict__ fc,
                               TypeTab tt, Phys<T> ph) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  int tl, tr, fl, frr;
  long long el, er;
  decode_fp(pl[i], tt, &tl, &el, &fl);
  decode_fp(pr[i], tt, &tr, &er, &frr);
  T ul[5], ur[5], ql[5], qr[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    long long il = fp_index(tt, tl, el, fl, 5, k);
    long long ir = fp_index(tt, tr, er, frr, 5, k);
    ul[k] = uf[il];
    ur[k] = uf[ir];
    ql[k] = q[il];
    qr[k] = q[ir];
  }
  T n[3] = {pn[4 * i], pn[4 * i + 1], pn[4 * i + 2]};
  T ml = pn[4 * i + 3], mr = pmr[i];
  T F[5];
  rusanov(ul, ur, n, ph, F);
  const T rl = ml / mr, rr = mr / ml;
  const T wl = T(0.5) + ph.beta, wr = T(0.5) - ph.beta;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const T G = F[k] + ph.tau * (ul[k] - ur[k]);
    fc[fp_index(tt, tl, el, fl, 5, k)] = ml * G - (wl * ql[k] - wr * rl * qr[k]);
    fc[fp_index(tt, tr, er, frr, 5, k)] = -mr * G + (wl * rr * ql[k] - wr * qr[k]);
  }
}

// Boundary points: F^C = |S^T n~| Rus(u, ghost) - q (q already averaged).
// Exchange points take the partner's q (xq [nb][5]) and |S^T n~| (xm [nb])
// as an interior face does: F^C = m Rus - (q - (m / m_R) q_R) / 2.
template <typename T>
__global__ void k_bnd_flux_ns(int nb, const int32_t* __restrict__ bidx,
                              const int32_t* __restrict__ bbc,
                              const T* __restrict__ bn,
                              const T* __restrict__ uf,
                              const T* __restrict__ q, T* __restrict__ fc,
                              TypeTab tt, Phys<T> ph, BCTab<T> bc,
                              const T* __restrict__ xu = nullptr,
                              const T* __restrict__ xq = nullptr,
                              const T* __restrict__ xm = nullptr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int t, f;
  long long e;
  decode_fp(bidx[i], tt, &t, &e, &f);
  T ul[5], ur[5], n[3] = {bn[4 * i], bn[4 * i + 1], bn[4 * i + 2]};
#pragma unroll
  for (int k = 0; k < 5; ++k) ul[k] = uf[fp_index(tt, t, e, f, 5, k)];
  const int b = bbc[i];
  ghost_state_x(bc, b, i, xu, ul, ur);
  T F[5];
  rusanov(ul, ur, n, ph, F);
  T m = bn[4 * i + 3];
  if (bc.kind[b] == 2) {
    const T rl = m / xm[i];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      long long ix = fp_index(tt, t, e, f, 5, k);
      fc[ix] = m * (F[k] + ph.tau * (ul[k] - ur[k])) - T(0.5) * (q[ix] - rl * xq[5 * i + k]);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    long long ix = fp_index(tt, t, e, f, 5, k);
    fc[ix] = m * (F[k] + ph.tau * (ul[k] - ur[k])) - q[ix];
  }
}

// Halo exchange of one part: every exchange point it owns pushes its trace
// (nv values at the flux point: u, the gradient, or the viscous normal flux
// q) into the receive buffer of the part that shares the point, at that
// part's boundary-point slot.  dst[r] is part r's buffer ([nb_r][nv]).
template <typename T>
__global__ void k_exchange_push(int n, const int32_t* __restrict__ code,
                                const int32_t* __restrict__ to,
                                const int32_t* __restrict__ slot,
                                const T* __restrict__ src, int nv,
                                T* const* __restrict__ dst, TypeTab tt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t, f;
  long long e;
  decode_fp(code[i], tt, &t, &e, &f);
  T* d = dst[to[i]] + (long long)slot[i] * nv;
  for (int c = 0; c < nv; ++c) d[c] = src[fp_index(tt, t, e, f, nv, c)];
}

// Exchange with other processes: gather the traces (nv values per point) at
// the listed own exchange points into a message buffer [n][nv], and scatter
// a received buffer into the receive slots of the same points.
template <typename T>
__global__ void k_exchange_gather(int n, const int32_t* __restrict__ list,
                                  const int32_t* __restrict__ bidx,
                                  const T* __restrict__ src, int nv,
                                  T* __restrict__ dst, TypeTab tt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t, f;
  long long e;
  decode_fp(bidx[list[i]], tt, &t, &e, &f);
  for (int c = 0; c < nv; ++c) dst[(long long)i * nv + c] = src[fp_index(tt, t, e, f, nv, c)];
}

template <typename T>
__global__ void k_exchange_scatter(int n, const int32_t* __restrict__ list,
                                   const T* __restrict__ src, int nv,
                                   T* __restrict__ dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long slot = list[i];
  for (int c = 0; c < nv; ++c) dst[slot * nv + c] = src[(long long)i * nv + c];
}

// ---------------------------------------------------------------------------
// Dense kernels (prisms, tetrahedra, and the dense hexahedron variant) are
// persistent: each CTA copies the type's operators into shared memory once
// (when they fit) and then loops over groups of EPB elements.

// one point's row of 5 / 15 values (16-byte aligned rows)
template <typename T>
__device__ __forceinline__ void lds_row5(const T* p, T v[5]) {
  if constexpr (sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  v[4] = p[4];
}

template <typename T>
__device__ __forceinline__ void lds_row15(const T* p, T v[15]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float4 a = reinterpret_cast<const float4*>(p)[i];
      v[4 * i] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = a.z; v[4 * i + 3] = a.w;
    }
    const float4 a = reinterpret_cast<const float4*>(p)[3];
    v[12] = a.x; v[13] = a.y; v[14] = a.z;
  } else {
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      const double2 a = reinterpret_cast<const double2*>(p)[i];
      v[2 * i] = a.x; v[2 * i + 1] = a.y;
    }
    v[14] = p[14];
  }
}

template <typename T>
__device__ __forceinline__ void sts_row5(T* p, const T v[5]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
  p[4] = v[4];
}

template <typename T>
__device__ __forceinline__ void sts_row15(T* p, const T v[15]) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
      reinterpret_cast<float4*>(p)[i] =
          make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    reinterpret_cast<float4*>(p)[3] = make_float4(v[12], v[13], v[14], T(0));
  } else {
#pragma unroll
    for (int i = 0; i < 7; ++i)
      reinterpret_cast<double2*>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
    p[14] = v[14];
  }
}

// Per-element working arrays of the dense kernels.  FP32 (kRows): one row
// per point, the 5 variables of a point (row stride kP5 = 8) or its 15
// transformed-flux / gradient components (stride 16); the inner loops read
// a whole row with 128-bit shared loads (the same row for every thread of
// the element: a broadcast) instead of one 32-bit load per component, which
// relieves the shared-memory pipe that bounds the FP32 kernels.  FP64: one
// column per component ([5][n], [15][n]); the FP64 kernels are bound by the
// FP64 pipe and keep the skips of zero normal components.
template <typename T, int NU, int NF>
struct DenseLayout {
  static constexpr int kOps = 3 * NU * NU + 2 * NU * NF + 3 * NF;
  static constexpr bool kStaged = kOps * sizeof(T) <= 48 * 1024;
  static constexpr int kAlign = 16 / int(sizeof(T));
  static constexpr int kStagedCount = kStaged ? (kOps + kAlign - 1) / kAlign * kAlign : 0;
  static constexpr bool kRows = sizeof(T) == 4;
  static constexpr int kP5 = 8;
  static constexpr int kGradElem = kRows ? kP5 * NU + kP5 * NF + 16 * NU : 20 * NU + 5 * NF;
  static constexpr int kVolElem = kRows ? 16 * NU + kP5 * NF : 15 * NU + 5 * NF;
  // offsets of value (point q, component k) in a 5- / 15-component array
  // over n points
  template <int n>
  __device__ static constexpr int at5(int q, int k) { return kRows ? q * kP5 + k : k * n + q; }
  template <int n>
  __device__ static constexpr int at15(int q, int c) { return kRows ? q * 16 + c : c * n + q; }
};

// the 5 / 15 values of point q (kRows: one row, vector loads)
template <typename L, int n, typename T>
__device__ __forceinline__ void get5(const T* a, int q, T v[5]) {
  if constexpr (L::kRows) {
    lds_row5(a + q * L::kP5, v);
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = a[k * n + q];
  }
}

template <typename L, int n, typename T>
__device__ __forceinline__ void put5(T* a, int q, const T v[5]) {
  if constexpr (L::kRows) {
    sts_row5(a + q * L::kP5, v);
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k) a[k * n + q] = v[k];
  }
}

template <typename L, int n, typename T>
__device__ __forceinline__ void get15(const T* a, int q, T v[15]) {
  if constexpr (L::kRows) {
    lds_row15(a + q * 16, v);
  } else {
#pragma unroll
    for (int c = 0; c < 15; ++c) v[c] = a[c * n + q];
  }
}

template <typename L, int n, typename T>
__device__ __forceinline__ void put15(T* a, int q, const T v[15]) {
  if constexpr (L::kRows) {
    sts_row15(a + q * 16, v);
  } else {
#pragma unroll
    for (int c = 0; c < 15; ++c) a[c * n + q] = v[c];
  }
}

template <typename T, int NU, int NF>
__device__ __forceinline__ DenseOps<T> stage_dense_ops(const DenseOps<T>& g,
                                                       T* s) {
  if (!DenseLayout<T, NU, NF>::kStaged) return g;
  T* dt = s;
  T* m0 = dt + 3 * NU * NU;
  T* li = m0 + NU * NF;
  T* nr = li + NU * NF;
  for (int i = threadIdx.x; i < 3 * NU * NU; i += blockDim.x) dt[i] = g.DT[i];
  for (int i = threadIdx.x; i < NU * NF; i += blockDim.x) {
    m0[i] = g.M0T[i];
    li[i] = g.LIFTT[i];
  }
  for (int i = threadIdx.x; i < 3 * NF; i += blockDim.x) nr[i] = g.NREF[i];
  __syncthreads();
  return DenseOps<T>{m0, dt, li, nr, g.Mc, g.Mv, g.nm};
}

// NS gradient path: corrected reference gradient D u + LIFT (n~ du), physical
// gradient (1/J) S^T grad~ u at solution points, and its interpolation to
// the flux points.
template <typename T, int NU, int NF, int EPB, bool QV>
__global__ void __launch_bounds__(EPB* NU)
    k_grad_dense(long long ne, const T* __restrict__ u,
                 const T* __restrict__ du, const T* __restrict__ smat,
                 const T* __restrict__ rcpdjac, DenseOps<T> gops,
                 T* __restrict__ grad, ViscArgs<T> va, BCTab<T> bc,
                 Phys<T> ph) {
  using L = DenseLayout<T, NU, NF>;
  constexpr int P5 = L::kP5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const DenseOps<T> ops = stage_dense_ops<T, NU, NF>(gops, sm);
  T* buf = sm + L::kStagedCount;
  const int le = threadIdx.x / NU, z = threadIdx.x % NU;
  T* us = buf + le * L::kGradElem;             // u at the solution points
  T* ds = us + (L::kRows ? P5 * NU : 5 * NU);  // du at the flux points
  T* gs = ds + (L::kRows ? P5 * NF : 5 * NF);  // physical gradient (15)
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
      for (int q = 0; q < NU; ++q) {
        T uq[5];
        get5<L, NU>(us, q, uq);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          T w = ops.DT[(d * NU + q) * NU + z];
#pragma unroll
          for (int k = 0; k < 5; ++k) gref[d][k] += w * uq[k];
        }
      }
      for (int f = 0; f < NF; ++f) {
        const T l = ops.LIFTT[f * NU + z];
        T dq[5];
        get5<L, NF>(ds, f, dq);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T nd = ops.NREF[f * 3 + d];  // the same f on every thread
          if (nd != T(0)) {
            const T w = l * nd;
#pragma unroll
            for (int k = 0; k < 5; ++k) gref[d][k] += w * dq[k];
          }
        }
      }
      T S[3][3];
#pragma unroll
      for (int r = 0; r < 9; ++r) S[r / 3][r % 3] = smat[(e * 9 + r) * NU + z];
      T rj = rcpdjac[e * NU + z];
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
        if (ops.nm > 0) {  // M0 by its nonzeros
          for (int j = 0; j < ops.nm; ++j) {
            const T m = ops.Mv[f * ops.nm + j];
            T g[15];
            get15<L, NU>(gs, ops.Mc[f * ops.nm + j], g);
#pragma unroll
            for (int c = 0; c < 15; ++c) acc[c] += m * g[c];
          }
        } else {
          for (int q = 0; q < NU; ++q) {
            const T m = ops.M0T[q * NF + f];
            T g[15];
            get15<L, NU>(gs, q, g);
#pragma unroll
            for (int c = 0; c < 15; ++c) acc[c] += m * g[c];
          }
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

// ---------------------------------------------------------------------------
// Volume kernel: transformed flux f~ = S F at solution points, Eq. (FRfinal)
// divergence  sum_d D_d f~_d + LIFT (F^C - n~.M0 f~), negdivconf R = -div/J,
// the RK epilogue, and the next stage's u_f = M0 u_next.
// AA: f~ is the anti-aliased projection precomputed in tflux
// ([ne][3][5][NU], Section 3.2) and is read instead of collocated.
template <typename T, int NU, int NF, int EPB, bool NS, bool AA = false>
__global__ void __launch_bounds__(EPB* NU)
    k_vol_dense(long long ne, const T* __restrict__ u,
                const T* __restrict__ grad, const T* __restrict__ fc,
                const T* __restrict__ smat, const T* __restrict__ rcpdjac,
                DenseOps<T> gops, Phys<T> ph, StageArgs<T> sa,
                const T* __restrict__ tflux = nullptr) {
  using L = DenseLayout<T, NU, NF>;
  constexpr int P5 = L::kP5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const DenseOps<T> ops = stage_dense_ops<T, NU, NF>(gops, sm);
  T* buf = sm + L::kStagedCount;
  const int le = threadIdx.x / NU, z = threadIdx.x % NU;
  T* ft = buf + le * L::kVolElem;  // f~ (component d * 5 + k), then u_next
  T* jm = ft + (L::kRows ? 16 * NU : 15 * NU);  // F^C - n~.f~ at the flux points
  const long long ngroups = (ne + EPB - 1) / EPB;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long long e = grp * EPB + le;
    const bool act = e < ne;
    T uz[5];
    if (act) {
#pragma unroll
      for (int k = 0; k < 5; ++k) uz[k] = u[(e * 5 + k) * NU + z];
    }
    if (AA && act) {
      T fv[15];
#pragma unroll
      for (int c = 0; c < 15; ++c) fv[c] = tflux[(e * 15 + c) * NU + z];
      put15<L, NU>(ft, z, fv);
    } else if (act) {
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
      for (int f = z; f < NF; f += NU) {
        T fn[5] = {0, 0, 0, 0, 0};
        const T nr0 = ops.NREF[f * 3], nr1 = ops.NREF[f * 3 + 1], nr2 = ops.NREF[f * 3 + 2];
        for (int j = 0; j < ops.nm; ++j) {  // M0 by its nonzeros
          const T m = ops.Mv[f * ops.nm + j];
          T v[15];
          get15<L, NU>(ft, ops.Mc[f * ops.nm + j], v);
          const T w0 = m * nr0, w1 = m * nr1, w2 = m * nr2;
#pragma unroll
          for (int k = 0; k < 5; ++k) fn[k] += w0 * v[k] + w1 * v[5 + k] + w2 * v[10 + k];
        }
        for (int q = 0; q < (ops.nm > 0 ? 0 : NU); ++q) {
          const T m = ops.M0T[q * NF + f];
          if constexpr (L::kRows) {
            T v[15];
            lds_row15(ft + q * 16, v);
            const T w0 = m * nr0, w1 = m * nr1, w2 = m * nr2;
#pragma unroll
            for (int k = 0; k < 5; ++k) fn[k] += w0 * v[k] + w1 * v[5 + k] + w2 * v[10 + k];
          } else {
            const T nr[3] = {nr0, nr1, nr2};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              if (nr[d] == T(0)) continue;
              const T w = m * nr[d];
#pragma unroll
              for (int k = 0; k < 5; ++k) fn[k] += w * ft[(d * 5 + k) * NU + q];
            }
          }
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
      for (int q = 0; q < NU; ++q) {
        T v[15];
        get15<L, NU>(ft, q, v);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T w = ops.DT[(d * NU + q) * NU + z];
#pragma unroll
          for (int k = 0; k < 5; ++k) div[k] += w * v[d * 5 + k];
        }
      }
      for (int f = 0; f < NF; ++f) {
        const T l = ops.LIFTT[f * NU + z];
        T jv[5];
        get5<L, NF>(jm, f, jv);
#pragma unroll
        for (int k = 0; k < 5; ++k) div[k] += l * jv[k];
      }
      T rj = rcpdjac[e * NU + z];
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
          for (int j = 0; j < ops.nm; ++j) {  // M0 by its nonzeros
            const T m = ops.Mv[f * ops.nm + j];
            T v[5];
            get5<L, NU>(ft, ops.Mc[f * ops.nm + j], v);
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[k] += m * v[k];
          }
          for (int q = 0; q < (ops.nm > 0 ? 0 : NU); ++q) {
            const T m = ops.M0T[q * NF + f];
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
