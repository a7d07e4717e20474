// Pointwise compressible Euler / Navier-Stokes physics on the device.
//
// Conserved variables u = (rho, rho u, rho v, rho w, E): the field index
// alpha of Eq. (gov) of the paper (Section 2).  The paper names the
// compressible Euler and Navier-Stokes solvers without printing their
// formulas; these are the standard nondimensional forms:
//   p = (gamma-1)(E - rho|v|^2/2)
//   inviscid flux F_j = (rho v_j, rho v v_j + p e_j, (E+p) v_j)
//   viscous flux (subtracted) (0, tau_.j, v.tau_.j + kappa de/dx_j),
//   tau = mu(grad v + grad v^T - 2/3 div v I), e = E/rho - |v|^2/2,
//   kappa = mu gamma / Pr
//   Rusanov common flux (Eq. comm_flux):
//   (F(u-)+F(u+)).n/2 - lambda (u+ - u-)/2,
//   lambda = max(|v-.n| + c-, |v+.n| + c+).
#pragma once
#include <cuda_runtime.h>

namespace frgb {

// beta, tau: LDG bias and penalty of the viscous coupling (0, 0: BR1)
template <typename T>
struct Phys {
  T gamma, gm1, mu, kappa;
  T beta = T(0), tau = T(0);
};

template <typename T>
__device__ __forceinline__ T fr_sqrt(T x);
template <>
__device__ __forceinline__ double fr_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float fr_sqrt<float>(float x) { return sqrtf(x); }

// normal inviscid flux n.F(u), pressure and normal velocity
template <typename T>
__device__ __forceinline__ void normal_flux(const T u[5], const T n[3],
                                            const Phys<T>& ph, T fn[5], T* c,
                                            T* vn) {
  T ri = T(1) / u[0];
  T vx = u[1] * ri, vy = u[2] * ri, vz = u[3] * ri;
  T p = ph.gm1 * (u[4] - T(0.5) * (u[1] * vx + u[2] * vy + u[3] * vz));
  T v = vx * n[0] + vy * n[1] + vz * n[2];
  fn[0] = u[0] * v;
  fn[1] = u[1] * v + p * n[0];
  fn[2] = u[2] * v + p * n[1];
  fn[3] = u[3] * v + p * n[2];
  fn[4] = (u[4] + p) * v;
  *c = fr_sqrt<T>(ph.gamma * p * ri);
  *vn = v;
}

template <typename T>
__device__ __forceinline__ void rusanov(const T ul[5], const T ur[5],
                                        const T n[3], const Phys<T>& ph,
                                        T F[5]) {
  T fl[5], fr[5], cl, cr, vl, vr;
  normal_flux(ul, n, ph, fl, &cl, &vl);
  normal_flux(ur, n, ph, fr, &cr, &vr);
  T a = fabs(vl) + cl, b = fabs(vr) + cr;
  T lam = a > b ? a : b;
#pragma unroll
  for (int k = 0; k < 5; ++k)
    F[k] = T(0.5) * (fl[k] + fr[k]) - T(0.5) * lam * (ur[k] - ul[k]);
}

// inviscid flux F[j][k] in direction j of variable k
template <typename T>
__device__ __forceinline__ void euler_flux(const T u[5], const Phys<T>& ph,
                                           T F[3][5]) {
  T ri = T(1) / u[0];
  T v[3] = {u[1] * ri, u[2] * ri, u[3] * ri};
  T p = ph.gm1 * (u[4] - T(0.5) * (u[1] * v[0] + u[2] * v[1] + u[3] * v[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    F[j][0] = u[1 + j];
    F[j][1] = u[1] * v[j];
    F[j][2] = u[2] * v[j];
    F[j][3] = u[3] * v[j];
    F[j][1 + j] += p;
    F[j][4] = (u[4] + p) * v[j];
  }
}

// viscous flux from u and its physical gradient g[j][k] = du_k/dx_j;
// accumulates  F[j][k] += sgn * Fv[j][k]
template <typename T>
__device__ __forceinline__ void viscous_flux_acc(const T u[5], const T g[3][5],
                                                 const Phys<T>& ph, T sgn,
                                                 T F[3][5]) {
  T ri = T(1) / u[0];
  T v[3] = {u[1] * ri, u[2] * ri, u[3] * ri};
  T er = u[4] * ri;
  T gv[3][3], ge[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int i = 0; i < 3; ++i) gv[j][i] = (g[j][1 + i] - v[i] * g[j][0]) * ri;
    ge[j] = (g[j][4] - er * g[j][0]) * ri -
            (v[0] * gv[j][0] + v[1] * gv[j][1] + v[2] * gv[j][2]);
  }
  T div = gv[0][0] + gv[1][1] + gv[2][2];
  T mu = ph.mu;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    T tau[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) tau[i] = mu * (gv[j][i] + gv[i][j]);
    tau[j] -= T(2.0 / 3.0) * mu * div;
    F[j][1] += sgn * tau[0];
    F[j][2] += sgn * tau[1];
    F[j][3] += sgn * tau[2];
    F[j][4] += sgn * (v[0] * tau[0] + v[1] * tau[1] + v[2] * tau[2] +
                      ph.kappa * ge[j]);
  }
}

// normal viscous flux n.Fv accumulated into f[k] with sign sgn, formed
// directly: (tau n)_i = mu (sum_j (dv_i/dx_j + dv_j/dx_i) n_j - 2/3 div v n_i),
// energy v.(tau n) + kappa n.grad e (the full tensor is never built).
template <typename T>
__device__ __forceinline__ void viscous_normal_acc(const T u[5],
                                                   const T g[3][5],
                                                   const T n[3],
                                                   const Phys<T>& ph, T sgn,
                                                   T f[5]) {
  const T ri = T(1) / u[0];
  const T v[3] = {u[1] * ri, u[2] * ri, u[3] * ri};
  const T er = u[4] * ri;
  T gv[3][3];  // gv[j][i] = d v_i / d x_j
  T gen = T(0);  // n . grad e
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int i = 0; i < 3; ++i) gv[j][i] = (g[j][1 + i] - v[i] * g[j][0]) * ri;
    const T ge = (g[j][4] - er * g[j][0]) * ri -
                 (v[0] * gv[j][0] + v[1] * gv[j][1] + v[2] * gv[j][2]);
    gen += n[j] * ge;
  }
  const T div23 = T(2.0 / 3.0) * (gv[0][0] + gv[1][1] + gv[2][2]);
  T tn[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T s = -div23 * n[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) s += (gv[j][i] + gv[i][j]) * n[j];
    tn[i] = ph.mu * s;
  }
  f[1] += sgn * tn[0];
  f[2] += sgn * tn[1];
  f[3] += sgn * tn[2];
  f[4] += sgn * (v[0] * tn[0] + v[1] * tn[1] + v[2] * tn[2] + ph.kappa * gen);
}

}  // namespace frgb
