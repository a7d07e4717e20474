"""Compressible Euler / Navier-Stokes physics for the oracle (test infra only).

Conserved variables u = (rho, rho u, rho v, rho w, E), the field index alpha
of Eq. (gov).  The paper names the compressible Euler and Navier-Stokes
solvers but prints none of their formulas; these are the textbook
(nondimensional) forms:

* p = (gamma - 1) (E - rho |v|^2 / 2)
* inviscid flux F_j = (rho v_j, rho v v_j + p e_j, (E + p) v_j)
* viscous flux (subtracted): (0, tau_.j, v . tau_.j + kappa de/dx_j) with
  tau = mu (grad v + grad v^T - 2/3 div v I), e = E/rho - |v|^2/2 and
  kappa = mu gamma / Pr (internal-energy form of Fourier's law, c_v = 1)
* Rusanov common flux for Eq. (comm_flux):
  F = (F(u-) + F(u+)).n / 2 - lambda (u+ - u-) / 2,
  lambda = max(|v- . n| + c-, |v+ . n| + c+), n the physical unit normal.

Arrays carry the variable index last; fluxes are (..., 3, 5) with the
spatial direction before the variable.
"""
import numpy as np


def primitives(u, gamma):
    rho = u[..., 0]
    v = u[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (u[..., 4] - 0.5 * rho * np.sum(v * v, axis=-1))
    return rho, v, p


def euler_flux(u, gamma):
    rho, v, p = primitives(u, gamma)
    F = np.empty(u.shape[:-1] + (3, 5))
    for j in range(3):
        F[..., j, 0] = u[..., 1 + j]
        for i in range(3):
            F[..., j, 1 + i] = u[..., 1 + i] * v[..., j]
        F[..., j, 1 + j] += p
        F[..., j, 4] = (u[..., 4] + p) * v[..., j]
    return F


def viscous_flux(u, gu, gamma, mu, pr):
    """Viscous flux from u (..., 5) and its physical gradient (..., 3, 5)."""
    rho = u[..., 0]
    v = u[..., 1:4] / rho[..., None]
    E = u[..., 4]
    # grad v[..., j, i] = d v_i / d x_j
    gv = (gu[..., :, 1:4] - v[..., None, :] * gu[..., :, 0:1]) / rho[..., None, None]
    ge = ((gu[..., :, 4] - (E / rho)[..., None] * gu[..., :, 0]) / rho[..., None]
          - np.einsum("...i,...ji->...j", v, gv))
    div = np.einsum("...ii->...", gv)
    tau = mu * (gv + np.swapaxes(gv, -1, -2))
    for i in range(3):
        tau[..., i, i] -= 2.0 / 3.0 * mu * div
    kappa = mu * gamma / pr
    F = np.zeros(u.shape[:-1] + (3, 5))
    F[..., :, 1:4] = tau
    F[..., :, 4] = np.einsum("...i,...ji->...j", v, tau) + kappa * ge
    return F


def rusanov(ul, ur, n, gamma):
    """Common normal flux across a face with unit normal n (from ul side)."""
    fl = np.einsum("...j,...jv->...v", n, euler_flux(ul, gamma))
    fr = np.einsum("...j,...jv->...v", n, euler_flux(ur, gamma))
    rl, vl, pl = primitives(ul, gamma)
    rr, vr, pr_ = primitives(ur, gamma)
    cl = np.sqrt(gamma * pl / rl)
    cr = np.sqrt(gamma * pr_ / rr)
    lam = np.maximum(np.abs(np.sum(vl * n, axis=-1)) + cl,
                     np.abs(np.sum(vr * n, axis=-1)) + cr)
    return 0.5 * (fl + fr) - 0.5 * lam[..., None] * (ur - ul)


def prim_to_cons(rho, v, p, gamma):
    u = np.empty(np.shape(rho) + (5,))
    u[..., 0] = rho
    u[..., 1:4] = rho[..., None] * v
    u[..., 4] = p / (gamma - 1.0) + 0.5 * rho * np.sum(v * v, axis=-1)
    return u
