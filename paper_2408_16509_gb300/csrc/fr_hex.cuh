// Sum-factorised hexahedron kernels (PyFR v2.0.3, Section 2, Eqs. disu and
// FRfinal, on tensor-product elements).
//
// The hexahedron's operators are Kronecker products of 1D factors on the
// N = p+1 Gauss-Legendre points: interpolation to a face is one
// N-point dot product along the line normal to it, the derivative along
// x~_d is the 1D derivative matrix along the d-lines, and the DG correction
// of a face point touches only the N solution points of its line, with
// weights g_R'(x_a) (plus face) and -g_L'(x_a) (minus face) (Huynh 2007).
// This is the "bespoke kernel that elides multiplications by zero" idea of
// the paper's matrix-multiplication paragraph, done by construction.
//
// Thread mapping: one thread per solution point (a, b, c), point index
// a + N b + N^2 c; blockDim.x / NU elements per CTA (at most EPB, the
// launch bound; the autotuner picks the tile).  Flux point index
// face * N^2 + i + N j, faces x-, x+, y-, y+, z-, z+ with (i, j) the two
// tangential indices in (y,z), (x,z), (x,y) order.
#pragma once
#include "fr_kernels.cuh"

namespace frgb {

template <typename T>
struct HexOps {
  T d1[8][8];  // d1[a][m] = l_m'(x_a)
  T lm[8], lp[8];  // l_m(-1), l_m(+1)
  T gl[8], gr[8];  // correction weights of the minus / plus face
  T xg[8];         // the line points themselves
  int gather;      // 1: Gauss-Lobatto lines, the face points are the line
                   //    end points (interpolation to a face is a copy)
};

// register type used for the RK solution / accumulator registers
template <typename T, typename TR>
struct HexStage {
  int mode, stage;
  TR* X;
  TR* A;
  T* Y;
  T* out;
  const double* dt;
  int* flag;
  T* uf_next;
  TR* E = nullptr;  // embedded-error register of an adaptive step (or nullptr)
};

template <int N>
__device__ __forceinline__ int fp_of(int face, int i, int j) {
  return face * N * N + i + N * j;
}

// solution point of face point (face, i, j) at position m along its line
template <int N>
__device__ __forceinline__ int line_pt(int face, int i, int j, int m) {
  int dir = face >> 1;
  if (dir == 0) return m + N * i + N * N * j;
  if (dir == 1) return i + N * m + N * N * j;
  return i + N * j + N * N * m;
}

// Which RK registers the stage update reads: X (nx) and A (na).
template <typename T, typename TR>
__device__ __forceinline__ void hex_stage_needs(const HexStage<T, TR>& a, bool* nx,
                                                bool* na) {
  *nx = a.mode == 2 || (a.mode == 1 && a.stage < 3);
  *na = a.mode == 1 && a.stage > 0;
}

// The mixed form's RK epilogue (FP32 stage values and right-hand side, FP64
// registers): each increment c dt r is formed in FP32 (r carries FP32
// rounding already) and added to the FP64 register exactly as a double, and
// the next stage value is the register rounded to FP32 plus its FP32
// increment.  One FP64 instruction per register write; the conversions run
// on the integer pipe.  Modes 1 and 2 as in hex_stage_apply.
template <typename T, typename TR>
__device__ __forceinline__ void hex_stage_apply_mixed(const HexStage<T, TR>& a,
                                                      long long i0, long long vstr,
                                                      const T R[5], const TR x[5],
                                                      const TR ac[5], T s[5]) {
  const float dt = narrow_f64(*a.dt);
  const int st = a.stage;
  if (a.mode == 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const long long i = i0 + k * vstr;
      const float r = R[k];
      if (st == 0) {
        a.A[i] = x[k] + widen_f32(dt * (1.0f / 6.0f) * r);
        const float y = narrow_f64(x[k]) + dt * 0.5f * r;
        a.Y[i] = y;
        s[k] = y;
      } else if (st < 3) {
        a.A[i] = ac[k] + widen_f32(dt * (1.0f / 3.0f) * r);
        const float y = narrow_f64(x[k]) + (st == 1 ? dt * 0.5f : dt) * r;
        a.Y[i] = y;
        s[k] = y;
      } else {
        const double xx = ac[k] + widen_f32(dt * (1.0f / 6.0f) * r);
        a.X[i] = xx;
        s[k] = narrow_f64(xx);
      }
    }
    return;
  }
  const float bdt = c_rk45_bf[st] * dt;
  const float adt = st < 4 ? (c_rk45_af[st] - c_rk45_bf[st]) * dt : 0.f;
  const float edt = c_rk45_ef[st] * dt;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const long long i = i0 + k * vstr;
    const float r = R[k];
    const double xx = x[k] + widen_f32(bdt * r);
    a.X[i] = xx;
    if (a.E) {  // error estimate dt sum_i (b_i - bhat_i) R_i
      const double ev = widen_f32(edt * r);
      a.E[i] = st == 0 ? ev : a.E[i] + ev;
    }
    const float xf = narrow_f64(xx);
    if (st < 4) {
      const float y = xf + adt * r;
      a.Y[i] = y;
      s[k] = y;
    } else {
      s[k] = xf;
    }
  }
}

// RK epilogue for one point from the register values x (X) and ac (A) read
// beforehand: R[5] -> registers; s receives the next stage value (u for a
// bare right-hand side, mode 0).
template <typename T, typename TR>
__device__ __forceinline__ void hex_stage_apply(const HexStage<T, TR>& a,
                                                long long i0, long long vstr,
                                                const T u[5], const T R[5],
                                                const TR x[5], const TR ac[5],
                                                T s[5]) {
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 5; ++k) bad |= !isfinite(R[k]);
  if (bad) atomicOr(a.flag, 1);
  if (a.mode == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      a.out[i0 + k * vstr] = R[k];
      s[k] = u[k];
    }
    return;
  }
  if constexpr (sizeof(T) == 4 && sizeof(TR) == 8) {
    hex_stage_apply_mixed(a, i0, vstr, R, x, ac, s);
    return;
  }
  const TR dt = TR(*a.dt);
  const int st = a.stage;
  if (a.mode == 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const long long i = i0 + k * vstr;
      const TR r = TR(R[k]);
      if (st == 0) {
        a.A[i] = x[k] + dt * TR(1.0 / 6.0) * r;
        const T y = T(x[k] + dt * TR(0.5) * r);
        a.Y[i] = y;
        s[k] = y;
      } else if (st < 3) {
        a.A[i] = ac[k] + dt * TR(1.0 / 3.0) * r;
        const T y = T(x[k] + (st == 1 ? dt * TR(0.5) : dt) * r);
        a.Y[i] = y;
        s[k] = y;
      } else {
        const TR xx = ac[k] + dt * TR(1.0 / 6.0) * r;
        a.X[i] = xx;
        s[k] = T(xx);
      }
    }
    return;
  }
  const TR b = TR(c_rk45_b[st]);
  const TR am = st < 4 ? TR(c_rk45_a[st]) - b : TR(0);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const long long i = i0 + k * vstr;
    const TR r = TR(R[k]);
    const TR xx = x[k] + b * dt * r;
    a.X[i] = xx;
    if (a.E) {  // error estimate dt sum_i (b_i - bhat_i) R_i
      const TR ev = TR(c_rk45_e[st]) * dt * r;
      a.E[i] = st == 0 ? ev : a.E[i] + ev;
    }
    if (st < 4) {
      const T y = T(xx + am * dt * r);
      a.Y[i] = y;
      s[k] = y;
    } else {
      s[k] = T(xx);
    }
  }
}

// Register values the stage update of one point reads, from global memory.
template <typename T, typename TR>
__device__ __forceinline__ void hex_stage_load(const HexStage<T, TR>& a,
                                               long long i0, long long vstr,
                                               TR x[5], TR ac[5]) {
  bool nx, na;
  hex_stage_needs(a, &nx, &na);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    x[k] = nx ? a.X[i0 + k * vstr] : TR(0);
    ac[k] = na ? a.A[i0 + k * vstr] : TR(0);
  }
}

template <typename T, typename TR>
__device__ __forceinline__ void hex_stage_update(const HexStage<T, TR>& a,
                                                 long long i0, long long vstr,
                                                 const T u[5], const T R[5],
                                                 T s[5]) {
  TR x[5], ac[5];
  hex_stage_load(a, i0, vstr, x, ac);
  hex_stage_apply(a, i0, vstr, u, R, x, ac, s);
}

// interpolate smem field src[v][pt] to face point fp (5 variables)
template <typename T, int N, int NV, typename Ops>
__device__ __forceinline__ void face_interp(const T* src, int fp, const Ops& op,
                                            T out[NV]) {
  const int NF1 = N * N;
  int face = fp / NF1, r = fp - face * NF1;
  int i = r % N, j = r / N;
  if (op.gather) {  // Gauss-Lobatto: the face point is a solution point
    const int q = line_pt<N>(face, i, j, (face & 1) ? N - 1 : 0);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = src[k * N * N * N + q];
    return;
  }
  const T* w = (face & 1) ? op.lp : op.lm;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = T(0);
#pragma unroll
  for (int m = 0; m < N; ++m) {
    int q = line_pt<N>(face, i, j, m);
    T c = w[m];
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] += c * src[k * N * N * N + q];
  }
}

// Both faces of direction dir at face position (i, j): their flux points
// lie on the same line of solution points, so one pass over the line's N
// points (shared-memory reads) gives both values (o0: minus face, o1: plus
// face) with the weights l_m(-1), l_m(+1).
template <typename T, int N, int NV, typename Ops>
__device__ __forceinline__ void face_interp_pair(const T* src, int dir, int i, int j,
                                                 const Ops& op, T o0[NV], T o1[NV]) {
  constexpr int NU = N * N * N;
  if (op.gather) {  // Gauss-Lobatto: the line's end points
    const int q0 = line_pt<N>(2 * dir, i, j, 0), q1 = line_pt<N>(2 * dir, i, j, N - 1);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      o0[k] = src[k * NU + q0];
      o1[k] = src[k * NU + q1];
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) o0[k] = o1[k] = T(0);
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const int q = line_pt<N>(2 * dir, i, j, m);
    const T cm = op.lm[m], cp = op.lp[m];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const T v = src[k * NU + q];
      o0[k] += cm * v;
      o1[k] += cp * v;
    }
  }
}

// ---------------------------------------------------------------------------
// NS gradients on hexahedra: corrected reference gradient, physical gradient
// at solution points, and its value at the flux points.
// QV: write the viscous normal flux q (5 per flux point, for the q-based
// interface kernel) instead of the 15 gradient components at flux points.
// Shared memory per element of k_hex_grad: u [5][NU], du [5][NF], physical
// gradient [15][NU], and for the q form the traces [5][NF] and S^T n~
// [3][NF] at the flux points (type T, 16-byte padded).
template <typename T, int N, bool QV>
__host__ __device__ constexpr int hex_grad_bytes_per_elem() {
  return ((20 * N * N * N + (QV ? 78 : 30) * N * N) * int(sizeof(T)) + 15) / 16 * 16;
}

// The q form (FP32 values) is bounded to 64 registers at 250 threads so that
// four CTAs fit on an SM (a few bytes spill; measured faster than three).
template <typename T, typename TR, int N, int EPB, bool QV>
__global__ void __launch_bounds__(EPB* N* N* N, (QV && EPB * N * N * N >= 250 ? 4 : 1))
    k_hex_grad(long long ne, const T* __restrict__ uin, const TR* __restrict__ X,
               const T* __restrict__ du, const T* __restrict__ smat,
               const T* __restrict__ rcpdjac, HexOps<T> op,
               T* __restrict__ grad, ViscArgs<T> va, BCTab<T> bc,
               Phys<T> ph) {
  constexpr int NU = N * N * N, NF = 6 * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int le = threadIdx.x / NU, z = threadIdx.x - le * NU;
  const long long e = (long long)blockIdx.x * (blockDim.x / NU) + le;
  T* us = reinterpret_cast<T*>(smem_raw + le * hex_grad_bytes_per_elem<T, N, QV>());
  T* ds = us + 5 * NU;
  T* gs = ds + 5 * NF;
  T* ufs = gs + 15 * NU;  // [5][NF] traces (q form)
  T* nvs = ufs + 5 * NF;  // [3][NF] S^T n~ (q form)
  const int a = z % N, b = (z / N) % N, c = z / (N * N);
  // the element's u, du (and the q form's inputs) arrive by cp.async while
  // the metric terms load into registers
  T S[3][3], rj = T(0);
  if (e < ne) {
    if (uin) {
      async_copy(us, uin + e * 5 * NU, 5 * NU * int(sizeof(T)), z, NU);
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k) us[k * NU + z] = T(X[(e * 5 + k) * NU + z]);
    }
    async_copy(ds, du + e * 5 * NF, 5 * NF * int(sizeof(T)), z, NU);
    if (QV) {
      async_copy(ufs, va.uf + e * 5 * NF, 5 * NF * int(sizeof(T)), z, NU);
      async_copy(nvs, va.fnv + e * 3 * NF, 3 * NF * int(sizeof(T)), z, NU);
    }
#pragma unroll
    for (int r = 0; r < 9; ++r) S[r / 3][r % 3] = smat[(e * 9 + r) * NU + z];
    rj = rcpdjac[e * NU + z];
  }
  cp_async_wait_all();
  __syncthreads();
  if (e < ne) {
    T gref[3][5];
    const int N2 = N * N;
    T da[N], db[N], dc[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      da[m] = op.d1[a][m];
      db[m] = op.d1[b][m];
      dc[m] = op.d1[c][m];
    }
    const T gla = op.gl[a], gra = op.gr[a], glb = op.gl[b], grb = op.gr[b],
            glc = op.gl[c], grc = op.gr[c];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
      for (int m = 0; m < N; ++m) {
        gx += da[m] * us[k * NU + m + N * b + N2 * c];
        gy += db[m] * us[k * NU + a + N * m + N2 * c];
        gz += dc[m] * us[k * NU + a + N * b + N2 * m];
      }
      // correction: the face normal n~ is -e_d on the minus face
      gx += -gla * ds[k * NF + fp_of<N>(0, b, c)] +
            gra * ds[k * NF + fp_of<N>(1, b, c)];
      gy += -glb * ds[k * NF + fp_of<N>(2, a, c)] +
            grb * ds[k * NF + fp_of<N>(3, a, c)];
      gz += -glc * ds[k * NF + fp_of<N>(4, a, b)] +
            grc * ds[k * NF + fp_of<N>(5, a, b)];
      gref[0][k] = gx;
      gref[1][k] = gy;
      gref[2][k] = gz;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        T g = rj * (S[0][j] * gref[0][k] + S[1][j] * gref[1][k] +
                    S[2][j] * gref[2][k]);
        grad[(e * 15 + j * 5 + k) * NU + z] = g;
        gs[(j * 5 + k) * NU + z] = g;
      }
  }
  __syncthreads();
  if (e >= ne) return;
  // flux point f with its interpolated gradient g: q (q form) or g itself
  auto out = [&](int f, const T* g) {
    if (QV) {
      T u[5], G[3][5], nv[3], q[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) u[k] = ufs[k * NF + f];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        nv[j] = nvs[j * NF + f];
#pragma unroll
        for (int k = 0; k < 5; ++k) G[j][k] = g[j * 5 + k];
      }
      visc_q_pre(bc, ph, u, G, nv, int(va.fbc[e * NF + f]), q,
                 prescribed_at(va, e, f, NF));
#pragma unroll
      for (int k = 0; k < 5; ++k) va.q[(e * 5 + k) * NF + f] = q[k];
    } else {
#pragma unroll
      for (int k = 0; k < 15; ++k) va.q[(e * 15 + k) * NF + f] = g[k];
    }
  };
  if constexpr (sizeof(T) == 4) {
    // shared-memory bound: one thread per face pair (direction, position)
    for (int t = z; t < 3 * N * N; t += NU) {
      const int dir = t / (N * N), r = t - dir * N * N, i = r % N, j = r / N;
      T g0[15], g1[15];
      face_interp_pair<T, N, 15>(gs, dir, i, j, op, g0, g1);
      out(fp_of<N>(2 * dir, i, j), g0);
      out(fp_of<N>(2 * dir + 1, i, j), g1);
    }
  } else {
    // FP64-pipe bound: one thread per flux point spreads the arithmetic
    for (int f = z; f < NF; f += NU) {
      T g[15];
      face_interp<T, N, 15>(gs, f, op, g);
      out(f, g);
    }
  }
}

// ---------------------------------------------------------------------------
// Volume kernel on hexahedra: f~ = S F, divergence along the three line
// families, DG correction with the jump F^C - n~.f~ computed once per flux
// point, R = -div / J, RK epilogue and the next stage's u_f.
// Shared memory per element: f~ [3][5][NU] and F^C / jump [5][NF] (type T),
// then, for FP32 registers, the RK registers X, A [5][NU].  The element's
// F^C block (and those register blocks) are copied asynchronously
// (cp.async) at entry, so their loads overlap the flux arithmetic instead
// of following it.  FP64 registers are read directly: staging them would
// double the shared memory per element and cost more occupancy than the
// overlap gains.
template <typename T, int N>
__host__ __device__ constexpr int hex_vol_tbytes() {  // T part, 16-byte padded
  return ((15 * N * N * N + 30 * N * N) * int(sizeof(T)) + 15) / 16 * 16;
}

template <typename TR>
__host__ __device__ constexpr bool hex_vol_stage_regs() {
  return sizeof(TR) == 4;
}

template <typename T, typename TR, int N>
__host__ __device__ constexpr int hex_vol_bytes_per_elem() {
  return hex_vol_tbytes<T, N>() +
         (hex_vol_stage_regs<TR>() ? (10 * N * N * N * int(sizeof(TR)) + 15) / 16 * 16 : 0);
}

// AA: f~ is the anti-aliased projection precomputed in tflux
// ([ne][3][5][NU], Section 3.2) and is copied in instead of collocated.
template <typename T, typename TR, int N, int EPB, bool NS, bool AA = false>
__global__ void __launch_bounds__(EPB* N* N* N)
    k_hex_vol(long long ne, const T* __restrict__ uin, const T* __restrict__ grad,
              const T* __restrict__ fc, const T* __restrict__ smat,
              const T* __restrict__ rcpdjac, HexOps<T> op, Phys<T> ph,
              HexStage<T, TR> sa, const T* __restrict__ tflux = nullptr) {
  constexpr int NU = N * N * N, NF = 6 * N * N, N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int le = threadIdx.x / NU, z = threadIdx.x - le * NU;
  const long long e = (long long)blockIdx.x * (blockDim.x / NU) + le;
  unsigned char* eb = smem_raw + le * hex_vol_bytes_per_elem<T, TR, N>();
  T* ft = reinterpret_cast<T*>(eb);       // [3][5][NU]
  T* jm = ft + 15 * NU;                   // [5][NF]: F^C, then the jump
  TR* xs = reinterpret_cast<TR*>(eb + hex_vol_tbytes<T, N>());  // [5][NU]
  TR* as = xs + 5 * NU;                         // [5][NU]
  const int a = z % N, b = (z / N) % N, c = z / N2;
  bool nx, na;
  hex_stage_needs(sa, &nx, &na);
  constexpr bool SR = hex_vol_stage_regs<TR>();
  if (e < ne) {
    async_copy(jm, fc + e * 5 * NF, 5 * NF * int(sizeof(T)), z, NU);
    if (AA) async_copy(ft, tflux + e * 15 * NU, 15 * NU * int(sizeof(T)), z, NU);
    if (SR && nx) async_copy(xs, sa.X + e * 5 * NU, 5 * NU * int(sizeof(TR)), z, NU);
    if (SR && na) async_copy(as, sa.A + e * 5 * NU, 5 * NU * int(sizeof(TR)), z, NU);
  }
  T uz[5];
  if (e < ne) {
#pragma unroll
    for (int k = 0; k < 5; ++k)
      uz[k] = uin ? uin[(e * 5 + k) * NU + z] : T(sa.X[(e * 5 + k) * NU + z]);
  }
  if (!AA && e < ne) {
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
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int k = 0; k < 5; ++k)
        ft[(d * 5 + k) * NU + z] =
            S[d][0] * F[0][k] + S[d][1] * F[1][k] + S[d][2] * F[2][k];
  }
  cp_async_wait_all();
  __syncthreads();
  if (e < ne) {
    // jump at every flux point: F^C - n~ . M0 f~ (only the normal direction,
    // -e_dir on the minus face, +e_dir on the plus face); FP32: per face
    // pair (fewer shared reads), FP64: per flux point
    if constexpr (sizeof(T) == 4) {
      for (int t = z; t < 3 * N2; t += NU) {
        const int dir = t / N2, r = t - dir * N2, i = r % N, j = r / N;
        T f0[5], f1[5];
        face_interp_pair<T, N, 5>(ft + dir * 5 * NU, dir, i, j, op, f0, f1);
        const int fm = fp_of<N>(2 * dir, i, j), fp = fp_of<N>(2 * dir + 1, i, j);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          jm[k * NF + fm] = jm[k * NF + fm] + f0[k];
          jm[k * NF + fp] = jm[k * NF + fp] - f1[k];
        }
      }
    } else {
      for (int f = z; f < NF; f += NU) {
        int face = f / N2;
        int dir = face >> 1;
        T fn[5];
        face_interp<T, N, 5>(ft + dir * 5 * NU, f, op, fn);
        T sgn = (face & 1) ? T(1) : T(-1);
#pragma unroll
        for (int k = 0; k < 5; ++k) jm[k * NF + f] = jm[k * NF + f] - sgn * fn[k];
      }
    }
  }
  __syncthreads();
  T s[5];
  if (e < ne) {
    T R[5];
    const T rj = rcpdjac[e * NU + z];
    T da[N], db[N], dc[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      da[m] = op.d1[a][m];
      db[m] = op.d1[b][m];
      dc[m] = op.d1[c][m];
    }
    const T gla = op.gl[a], gra = op.gr[a], glb = op.gl[b], grb = op.gr[b],
            glc = op.gl[c], grc = op.gr[c];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const T* fx = ft + (0 * 5 + k) * NU;
      const T* fy = ft + (1 * 5 + k) * NU;
      const T* fz = ft + (2 * 5 + k) * NU;
      T dv = T(0);
#pragma unroll
      for (int m = 0; m < N; ++m) {
        dv += da[m] * fx[m + N * b + N2 * c];
        dv += db[m] * fy[a + N * m + N2 * c];
        dv += dc[m] * fz[a + N * b + N2 * m];
      }
      const T* jk = jm + k * NF;
      dv += gla * jk[fp_of<N>(0, b, c)] + gra * jk[fp_of<N>(1, b, c)];
      dv += glb * jk[fp_of<N>(2, a, c)] + grb * jk[fp_of<N>(3, a, c)];
      dv += glc * jk[fp_of<N>(4, a, b)] + grc * jk[fp_of<N>(5, a, b)];
      R[k] = -dv * rj;
    }
    TR xr[5], ar[5];
    if (SR) {
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        xr[k] = nx ? xs[k * NU + z] : TR(0);
        ar[k] = na ? as[k * NU + z] : TR(0);
      }
    } else {
      hex_stage_load(sa, e * 5 * NU + z, NU, xr, ar);
    }
    hex_stage_apply(sa, e * 5 * NU + z, NU, uz, R, xr, ar, s);
  }
  if (sa.uf_next == nullptr) return;
  __syncthreads();
  if (e < ne) {
#pragma unroll
    for (int k = 0; k < 5; ++k) ft[k * NU + z] = s[k];
  }
  __syncthreads();
  if (e >= ne) return;
  if constexpr (sizeof(T) == 4) {
    for (int t = z; t < 3 * N2; t += NU) {
      const int dir = t / N2, r = t - dir * N2, i = r % N, j = r / N;
      T v0[5], v1[5];
      face_interp_pair<T, N, 5>(ft, dir, i, j, op, v0, v1);
      const int fm = fp_of<N>(2 * dir, i, j), fp = fp_of<N>(2 * dir + 1, i, j);
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        sa.uf_next[(e * 5 + k) * NF + fm] = v0[k];
        sa.uf_next[(e * 5 + k) * NF + fp] = v1[k];
      }
    }
  } else {
    for (int f = z; f < NF; f += NU) {
      T v[5];
      face_interp<T, N, 5>(ft, f, op, v);
#pragma unroll
      for (int k = 0; k < 5; ++k) sa.uf_next[(e * 5 + k) * NF + f] = v[k];
    }
  }
}

// Eq. (disu) on hexahedra from the solution register.
template <typename T, typename TR, int N, int EPB>
__global__ void __launch_bounds__(EPB* N* N* N)
    k_hex_interp(long long ne, const TR* __restrict__ X, HexOps<T> op,
                 T* __restrict__ uf) {
  constexpr int NU = N * N * N, NF = 6 * N * N;
  __shared__ T us[EPB][5 * NU];
  const int le = threadIdx.x / NU, z = threadIdx.x - le * NU;
  const long long e = (long long)blockIdx.x * EPB + le;
  if (e < ne) {
#pragma unroll
    for (int k = 0; k < 5; ++k) us[le][k * NU + z] = T(X[(e * 5 + k) * NU + z]);
  }
  __syncthreads();
  if (e >= ne) return;
  for (int f = z; f < NF; f += NU) {
    T v[5];
    face_interp<T, N, 5>(us[le], f, op, v);
#pragma unroll
    for (int k = 0; k < 5; ++k) uf[(e * 5 + k) * NF + f] = v[k];
  }
}

}  // namespace frgb

namespace frgb {

// ---------------------------------------------------------------------------
// Variants for FP32 values (FP32 and mixed precision), where the path is
// bound by DRAM traffic rather than arithmetic: the metric terms of linear
// hexahedra are computed on the fly from the 8 vertices (24 numbers per
// element instead of 10 per solution point, Section 3.4 of the paper), and
// the volume kernel recomputes the corrected gradient from u and the
// flux-point jumps instead of reading 15 stored components per point.

// S = det(J) J^{-1} (rows a_j x a_k) and det J of the trilinear map at
// reference point x, vertices relative to vertex 0 (X[v][k]).
template <typename T>
__device__ __forceinline__ void hex_metric_at(const T* X, T x0, T x1, T x2,
                                              T S[3][3], T* det) {
  const int sg[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                        {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
  T a[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
  for (int v = 1; v < 8; ++v) {
    const T f0 = T(1) + T(sg[v][0]) * x0, f1 = T(1) + T(sg[v][1]) * x1,
            f2 = T(1) + T(sg[v][2]) * x2;
    const T d0 = T(0.125) * T(sg[v][0]) * f1 * f2;
    const T d1 = T(0.125) * T(sg[v][1]) * f0 * f2;
    const T d2 = T(0.125) * T(sg[v][2]) * f0 * f1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T xv = X[v * 3 + k];
      a[0][k] += d0 * xv;
      a[1][k] += d1 * xv;
      a[2][k] += d2 * xv;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T* b = a[(i + 1) % 3];
    const T* c = a[(i + 2) % 3];
    S[i][0] = b[1] * c[2] - b[2] * c[1];
    S[i][1] = b[2] * c[0] - b[0] * c[2];
    S[i][2] = b[0] * c[1] - b[1] * c[0];
  }
  *det = a[0][0] * S[0][0] + a[0][1] * S[0][1] + a[0][2] * S[0][2];
}

// reference coordinates of solution point (a,b,c) / flux point f
template <typename T, int N>
__device__ __forceinline__ void hex_fpt_ref(const HexOps<T>& op, const T* x1,
                                            int f, T x[3], T n[3]) {
  (void)op;
  const int face = f / (N * N), r = f - face * N * N;
  const int i = r % N, j = r / N, dir = face >> 1;
  const T side = (face & 1) ? T(1) : T(-1);
  const T s = x1[i], t = x1[j];
  if (dir == 0) { x[0] = side; x[1] = s; x[2] = t; }
  else if (dir == 1) { x[0] = s; x[1] = side; x[2] = t; }
  else { x[0] = s; x[1] = t; x[2] = side; }
  n[0] = n[1] = n[2] = T(0);
  n[dir] = side;
}

// corrected reference gradient at (a, b, c) from u (smem [5][NU]) and the
// flux-point jumps du (smem [5][NF])
template <typename T, int N, typename Ops>
__device__ __forceinline__ void hex_ref_grad(const T* us, const T* ds, const Ops& op,
                                             int a, int b, int c, T gref[3][5]) {
  constexpr int NU = N * N * N, NF = 6 * N * N, N2 = N * N;
  T da[N], db[N], dc[N];
#pragma unroll
  for (int m = 0; m < N; ++m) {
    da[m] = op.d1[a][m];
    db[m] = op.d1[b][m];
    dc[m] = op.d1[c][m];
  }
  const T gla = op.gl[a], gra = op.gr[a], glb = op.gl[b], grb = op.gr[b],
          glc = op.gl[c], grc = op.gr[c];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
    for (int m = 0; m < N; ++m) {
      gx += da[m] * us[k * NU + m + N * b + N2 * c];
      gy += db[m] * us[k * NU + a + N * m + N2 * c];
      gz += dc[m] * us[k * NU + a + N * b + N2 * m];
    }
    gx += -gla * ds[k * NF + fp_of<N>(0, b, c)] + gra * ds[k * NF + fp_of<N>(1, b, c)];
    gy += -glb * ds[k * NF + fp_of<N>(2, a, c)] + grb * ds[k * NF + fp_of<N>(3, a, c)];
    gz += -glc * ds[k * NF + fp_of<N>(4, a, b)] + grc * ds[k * NF + fp_of<N>(5, a, b)];
    gref[0][k] = gx;
    gref[1][k] = gy;
    gref[2][k] = gz;
  }
}

// Shared memory per element of the vertex-metric kernels (16-byte padded).
// Gradient: u [5][NU], du [5][NF], traces [5][NF], physical gradient
// [15][NU], vertices [24].  Volume: f~ [3][5][NU], F^C / jump [5][NF],
// u [5][NU], du [5][NF], vertices [24] (type T), then the
// RK registers X, A [5][NU] (type TR).
template <typename T, int N>
__host__ __device__ constexpr int hexv_grad_bytes_per_elem() {
  return ((20 * N * N * N + 60 * N * N + 24) * int(sizeof(T)) + 15) / 16 * 16;
}

template <typename T, int N>
__host__ __device__ constexpr int hexv_vol_tbytes() {
  return ((20 * N * N * N + 60 * N * N + 24) * int(sizeof(T)) + 15) / 16 * 16;
}

template <typename T, typename TR, int N>
__host__ __device__ constexpr int hexv_vol_bytes_per_elem() {
  return hexv_vol_tbytes<T, N>() + (10 * N * N * N * int(sizeof(TR)) + 15) / 16 * 16;
}

// NS gradients (FP32 values): vertex metrics, viscous flux at the flux
// points; nothing is stored at the solution points.  Every per-element
// input arrives by cp.async (the boundary tags of the thread's flux points
// and the vertices by plain loads).
template <typename T, typename TR, int N, int EPB>
__global__ void __launch_bounds__(EPB* N* N* N)
    k_hex_grad_v(long long ne, const T* __restrict__ uin, const TR* __restrict__ X,
                 const T* __restrict__ du, const T* __restrict__ verts,
                 HexOps<T> op, ViscArgs<T> va, BCTab<T> bc, Phys<T> ph) {
  constexpr int NU = N * N * N, NF = 6 * N * N, NFT = (NF + NU - 1) / NU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int le = threadIdx.x / NU, z = threadIdx.x - le * NU;
  const long long e = (long long)blockIdx.x * (blockDim.x / NU) + le;
  T* us = reinterpret_cast<T*>(smem_raw + le * hexv_grad_bytes_per_elem<T, N>());
  T* ds = us + 5 * NU;
  T* ufs = ds + 5 * NF;
  T* gs = ufs + 5 * NF;
  T* xv = gs + 15 * NU;  // the 24 vertex coordinates (relative to vertex 0)
  const int a = z % N, b = (z / N) % N, c = z / (N * N);
  int fb[NFT];
  if (e < ne) {
    if (uin) {
      async_copy(us, uin + e * 5 * NU, 5 * NU * int(sizeof(T)), z, NU);
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k) us[k * NU + z] = T(X[(e * 5 + k) * NU + z]);
    }
    async_copy(ds, du + e * 5 * NF, 5 * NF * int(sizeof(T)), z, NU);
    async_copy(ufs, va.uf + e * 5 * NF, 5 * NF * int(sizeof(T)), z, NU);
#pragma unroll
    for (int i = 0; i < NFT; ++i)
      fb[i] = z + i * NU < NF ? int(va.fbc[e * NF + z + i * NU]) : -1;
    if (z < 24) xv[z] = verts[e * 24 + z];
  }
  cp_async_wait_all();
  __syncthreads();
  if (e < ne) {
    T gref[3][5];
    hex_ref_grad<T, N>(us, ds, op, a, b, c, gref);
    T S[3][3], det;
    hex_metric_at(xv, op.xg[a], op.xg[b], op.xg[c], S, &det);
    const T rj = T(1) / det;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 5; ++k)
        gs[(j * 5 + k) * NU + z] =
            rj * (S[0][j] * gref[0][k] + S[1][j] * gref[1][k] + S[2][j] * gref[2][k]);
  }
  __syncthreads();
  if (e >= ne) return;
#pragma unroll
  for (int i = 0; i < NFT; ++i) {
    const int f = z + i * NU;
    if (f >= NF) break;
    T g[15];
    face_interp<T, N, 15>(gs, f, op, g);
    // S^T n~ at the flux point from the vertex map
    T xr[3], nr[3], nv[3];
    hex_fpt_ref<T, N>(op, op.xg, f, xr, nr);
    {
      T S[3][3], det;
      hex_metric_at(xv, xr[0], xr[1], xr[2], S, &det);
#pragma unroll
      for (int j = 0; j < 3; ++j) nv[j] = S[0][j] * nr[0] + S[1][j] * nr[1] + S[2][j] * nr[2];
    }
    T u[5], G[3][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) u[k] = ufs[k * NF + f];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 5; ++k) G[j][k] = g[j * 5 + k];
    T q[5] = {0, 0, 0, 0, 0};
    viscous_normal_acc(u, G, nv, ph, T(1), q);
    const int bb = fb[i];
    if (bb >= 0 && bc.kind[bb] != 2) {  // exchange points keep the inside q
      T ur[5], q2[5] = {0, 0, 0, 0, 0};
      const T* pre = prescribed_at(va, e, f, NF);
      if (bc.kind[bb] == 3 && pre) {
#pragma unroll
        for (int k = 0; k < 5; ++k) ur[k] = pre[k];
      } else {
        ghost_state(bc, bb, u, ur);
      }
      viscous_normal_acc(ur, G, nv, ph, T(1), q2);
#pragma unroll
      for (int k = 0; k < 5; ++k)
        q[k] = (T(0.5) + ph.beta) * q[k] + (T(0.5) - ph.beta) * q2[k];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) va.q[(e * 5 + k) * NF + f] = q[k];
  }
}

// Volume kernel (FP32 values): vertex metrics; for NS the corrected
// gradient is recomputed from u and du.  F^C, du and the RK registers
// arrive by cp.async while u and the vertices are loaded.
template <typename T, typename TR, int N, int EPB, bool NS>
__global__ void __launch_bounds__(EPB* N* N* N)
    k_hex_vol_v(long long ne, const T* __restrict__ uin, const T* __restrict__ du,
                const T* __restrict__ fc, const T* __restrict__ verts,
                HexOps<T> op, Phys<T> ph, HexStage<T, TR> sa) {
  constexpr int NU = N * N * N, NF = 6 * N * N, N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int le = threadIdx.x / NU, z = threadIdx.x - le * NU;
  const long long e = (long long)blockIdx.x * (blockDim.x / NU) + le;
  unsigned char* eb = smem_raw + le * hexv_vol_bytes_per_elem<T, TR, N>();
  T* ft = reinterpret_cast<T*>(eb);  // [3][5][NU]
  T* jm = ft + 15 * NU;              // [5][NF]: F^C, then the jump
  T* us = jm + 5 * NF;
  T* ds = us + 5 * NU;
  T* xv = ds + 5 * NF;  // the 24 vertex coordinates (relative to vertex 0)
  TR* xs = reinterpret_cast<TR*>(eb + hexv_vol_tbytes<T, N>());  // [5][NU]
  TR* as = xs + 5 * NU;                                          // [5][NU]
  const int a = z % N, b = (z / N) % N, c = z / N2;
  bool nx, na;
  hex_stage_needs(sa, &nx, &na);
  T uz[5];
  if (e < ne) {
    async_copy(jm, fc + e * 5 * NF, 5 * NF * int(sizeof(T)), z, NU);
    if (NS) async_copy(ds, du + e * 5 * NF, 5 * NF * int(sizeof(T)), z, NU);
    if (nx) async_copy(xs, sa.X + e * 5 * NU, 5 * NU * int(sizeof(TR)), z, NU);
    if (na) async_copy(as, sa.A + e * 5 * NU, 5 * NU * int(sizeof(TR)), z, NU);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      uz[k] = uin ? uin[(e * 5 + k) * NU + z] : T(sa.X[(e * 5 + k) * NU + z]);
      us[k * NU + z] = uz[k];
    }
    if (z < 24) xv[z] = verts[e * 24 + z];
  }
  cp_async_wait_all();
  __syncthreads();
  T rj = T(0);
  if (e < ne) {
    T S[3][3], det;
    hex_metric_at(xv, op.xg[a], op.xg[b], op.xg[c], S, &det);
    rj = T(1) / det;
    T F[3][5];
    euler_flux(uz, ph, F);
    if (NS) {
      T gref[3][5], g[3][5];
      hex_ref_grad<T, N>(us, ds, op, a, b, c, gref);
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 5; ++k)
          g[j][k] = rj * (S[0][j] * gref[0][k] + S[1][j] * gref[1][k] +
                          S[2][j] * gref[2][k]);
      viscous_flux_acc(uz, g, ph, T(-1), F);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int k = 0; k < 5; ++k)
        ft[(d * 5 + k) * NU + z] = S[d][0] * F[0][k] + S[d][1] * F[1][k] + S[d][2] * F[2][k];
  }
  __syncthreads();
  if (e < ne) {
    for (int f = z; f < NF; f += NU) {
      int face = f / N2;
      int dir = face >> 1;
      T fn[5];
      face_interp<T, N, 5>(ft + dir * 5 * NU, f, op, fn);
      T sgn = (face & 1) ? T(1) : T(-1);
#pragma unroll
      for (int k = 0; k < 5; ++k) jm[k * NF + f] = jm[k * NF + f] - sgn * fn[k];
    }
  }
  __syncthreads();
  T s[5];
  if (e < ne) {
    T R[5];
    T da[N], db[N], dc[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      da[m] = op.d1[a][m];
      db[m] = op.d1[b][m];
      dc[m] = op.d1[c][m];
    }
    const T gla = op.gl[a], gra = op.gr[a], glb = op.gl[b], grb = op.gr[b],
            glc = op.gl[c], grc = op.gr[c];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const T* fx = ft + (0 * 5 + k) * NU;
      const T* fy = ft + (1 * 5 + k) * NU;
      const T* fz = ft + (2 * 5 + k) * NU;
      T dv = T(0);
#pragma unroll
      for (int m = 0; m < N; ++m) {
        dv += da[m] * fx[m + N * b + N2 * c];
        dv += db[m] * fy[a + N * m + N2 * c];
        dv += dc[m] * fz[a + N * b + N2 * m];
      }
      const T* jk = jm + k * NF;
      dv += gla * jk[fp_of<N>(0, b, c)] + gra * jk[fp_of<N>(1, b, c)];
      dv += glb * jk[fp_of<N>(2, a, c)] + grb * jk[fp_of<N>(3, a, c)];
      dv += glc * jk[fp_of<N>(4, a, b)] + grc * jk[fp_of<N>(5, a, b)];
      R[k] = -dv * rj;
    }
    TR xr[5], ar[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      xr[k] = nx ? xs[k * NU + z] : TR(0);
      ar[k] = na ? as[k * NU + z] : TR(0);
    }
    hex_stage_apply(sa, e * 5 * NU + z, NU, uz, R, xr, ar, s);
  }
  if (sa.uf_next == nullptr) return;
  __syncthreads();
  if (e < ne) {
#pragma unroll
    for (int k = 0; k < 5; ++k) ft[k * NU + z] = s[k];
  }
  __syncthreads();
  if (e >= ne) return;
  for (int f = z; f < NF; f += NU) {
    T v[5];
    face_interp<T, N, 5>(ft, f, op, v);
#pragma unroll
    for (int k = 0; k < 5; ++k) sa.uf_next[(e * 5 + k) * NF + f] = v[k];
  }
}

}  // namespace frgb
