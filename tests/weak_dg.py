"""Nodal discontinuous Galerkin residual in weak form (test infrastructure;
imports nothing from ``oracle/`` or the library).

On affine hexahedra with Gauss-Legendre solution points, FR with the DG
correction function is the nodal DG method (Huynh 2007; the paper's
Eq. FRfinal with the DG choice of g).  This module computes that DG method
the other way round, as the weak form with Gauss-Legendre quadrature
collocated at the solution points:

  M_i du_i/dt = sum_q w_q |J| grad phi_i(x_q) . F(u_q)
                - sum_faces sum_f w_f |dA_f| phi_i(x_f) F^C_f,

with M_i = w_i |J| (the Gauss mass matrix is diagonal), grad phi_i the
physical gradient J^{-T} grad~ phi_i of the tensor Lagrange test function,
face quadrature at the face points and F^C the Rusanov common flux (plus,
for Navier-Stokes, minus the average of both sides' viscous fluxes).  BR1
gradients are the weak-form lift

  M_i theta_i = - sum_q w_q |J| grad phi_i(x_q) u_q
                + sum_faces sum_f w_f |dA_f| phi_i(x_f) u^C_f n_f.

Nothing here uses a correction function, a lift matrix or a reference
divergence: the two forms agree only if the FR pieces are right.  The 1D
Gauss rule is the Golub-Welsch eigenvalue construction.

Mesh: the block of parallelepipeds of ``brute_mp.spec_for`` (element
(i, j, k) = image of [2i, 2i+2] x [2j, 2j+2] x [2k, 2k+2] under x = A xi,
periodic in all three directions).
"""
import itertools

import numpy as np


def golub_welsch(n):
    k = np.arange(1, n)
    b = k / np.sqrt(4.0 * k * k - 1.0)
    x, V = np.linalg.eigh(np.diag(b, 1) + np.diag(b, -1))
    return x, 2.0 * V[0] ** 2


def lagrange_eval(xs, x):
    """L[q, m] = l_m(x_q) and dL[q, m] = l_m'(x_q), product formula."""
    x = np.atleast_1d(np.asarray(x, float))
    n = len(xs)
    L = np.ones((len(x), n))
    dL = np.zeros((len(x), n))
    for m in range(n):
        for k in range(n):
            if k == m:
                continue
            L[:, m] *= (x - xs[k]) / (xs[m] - xs[k])
        for j in range(n):
            if j == m:
                continue
            t = np.full(len(x), 1.0 / (xs[m] - xs[j]))
            for k in range(n):
                if k != m and k != j:
                    t *= (x - xs[k]) / (xs[m] - xs[k])
            dL[:, m] += t
    return L, dL


# ------------------------------------------------------------------ physics
def prim(u, gamma):
    rho = u[..., 0]
    v = u[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (u[..., 4] - 0.5 * np.sum(u[..., 1:4] * v, axis=-1))
    return rho, v, p


def euler_flux(u, gamma):
    """(..., 3 directions, 5 variables)."""
    rho, v, p = prim(u, gamma)
    F = u[..., None, :] * v[..., :, None]
    F[..., :, 1:4] += p[..., None, None] * np.eye(3)
    F[..., :, 4] += p[..., None] * v
    return F


def viscous_flux(u, g, gamma, mu, pr):
    """g[..., n, k] = d u_k / d x_n; primitive-variable form."""
    rho, v, p = prim(u, gamma)
    grho = g[..., :, 0]
    gv = (g[..., :, 1:4] - grho[..., :, None] * v[..., None, :]) / rho[..., None, None]
    gp = (gamma - 1.0) * (g[..., :, 4] - np.einsum("...i,...ni->...n", v, g[..., :, 1:4])
                          + 0.5 * np.sum(v * v, -1)[..., None] * grho)
    ge = (gp - p[..., None] * grho / rho[..., None]) / ((gamma - 1.0) * rho[..., None])
    div = np.trace(gv, axis1=-2, axis2=-1)
    tau = mu * (gv + np.swapaxes(gv, -1, -2)) - (2.0 / 3.0) * mu * div[..., None, None] * np.eye(3)
    F = np.zeros(u.shape[:-1] + (3, 5))
    F[..., :, 1:4] = tau
    F[..., :, 4] = np.einsum("...i,...ni->...n", v, tau) + mu * gamma / pr * ge
    return F


def rusanov(ul, ur, n, gamma):
    rl, vl, pl = prim(ul, gamma)
    rr, vr, pr_ = prim(ur, gamma)
    lam = np.maximum(np.abs(np.sum(vl * n, -1)) + np.sqrt(gamma * pl / rl),
                     np.abs(np.sum(vr * n, -1)) + np.sqrt(gamma * pr_ / rr))
    fl = np.einsum("...n,...nk->...k", n, euler_flux(ul, gamma))
    fr = np.einsum("...n,...nk->...k", n, euler_flux(ur, gamma))
    return 0.5 * (fl + fr) - 0.5 * lam[..., None] * (ur - ul)


# ------------------------------------------------------------------ DG
class WeakDG:
    def __init__(self, p, A, n, gamma=1.4, mu=0.0, pr=0.72):
        self.N = N = p + 1
        self.n = tuple(n)
        self.A = np.asarray(A, float)
        self.Ainv = np.linalg.inv(self.A)
        self.det = np.linalg.det(self.A)
        self.gamma, self.mu, self.pr = gamma, mu, pr
        x, w = golub_welsch(N)
        self.x1, self.w1 = x, w
        I = np.eye(N)
        _, dL = lagrange_eval(x, x)                       # dL[q, m]
        # point index a + N b + N^2 c; kron(C, B, A)[(c,b,a),(c',b',a')]
        dref = [np.kron(I, np.kron(I, dL)), np.kron(I, np.kron(dL, I)),
                np.kron(dL, np.kron(I, I))]               # [q, i]
        # physical gradient of test function i at point q, direction n
        self.gphi = np.einsum("dn,dqi->nqi", self.Ainv, np.stack(dref))
        self.W = np.kron(w, np.kron(w, w))
        self.M = self.W * self.det
        Lm, _ = lagrange_eval(x, -1.0)
        Lp, _ = lagrange_eval(x, 1.0)
        self.phi_face = {}
        for d, s in itertools.product(range(3), (-1, 1)):
            row = Lp if s > 0 else Lm                    # (1, N)
            mats = [I, I, I]
            mats[d] = row
            # tangential order (i, j) = the two other directions, lower first
            self.phi_face[(d, s)] = np.kron(mats[2], np.kron(mats[1], mats[0]))
        self.wface = np.kron(w, w)
        nvec = self.det * self.Ainv                       # row d: det J^{-T} e_d
        self.nmag = np.linalg.norm(nvec, axis=1)
        self.nunit = nvec / self.nmag[:, None]
        self.elems = list(itertools.product(*(range(k) for k in n)))

    def points(self):
        N = self.N
        out = {}
        for e in self.elems:
            for c, b, a in itertools.product(range(N), repeat=3):
                xi = np.array([self.x1[a], self.x1[b], self.x1[c]]) + 2 * np.array(e) + 1
                out[(e, a, b, c)] = self.A @ xi
        return out

    def _nb(self, e, d, s):
        f = list(e)
        f[d] = (f[d] + s) % self.n[d]
        return tuple(f)

    def rhs(self, u, physics="euler"):
        """u: {elem: (N^3, 5)} in point order a + N b + N^2 c."""
        g = self.gamma
        ns = physics == "ns"
        faces = list(itertools.product(range(3), (-1, 1)))
        tr = {(e, d, s): self.phi_face[(d, s)] @ u[e] for e in self.elems
              for d, s in faces}
        theta = None
        if ns:
            theta = {}
            for e in self.elems:
                vol = -np.einsum("q,nqi,qk->ink", self.W * self.det, self.gphi, u[e])
                for d, s in faces:
                    uc = 0.5 * (tr[(e, d, s)] + tr[(self._nb(e, d, s), d, -s)])
                    n = s * self.nunit[d]
                    vol += np.einsum("f,fi,fk,n->ink", self.wface * self.nmag[d],
                                     self.phi_face[(d, s)], uc, n)
                theta[e] = vol / self.M[:, None, None]
            gtr = {(e, d, s): np.einsum("fi,ink->fnk", self.phi_face[(d, s)], theta[e])
                   for e in self.elems for d, s in faces}
        out = {}
        for e in self.elems:
            F = euler_flux(u[e], g)
            if ns:
                F = F - viscous_flux(u[e], theta[e], g, self.mu, self.pr)
            res = np.einsum("q,nqi,qnk->ik", self.W * self.det, self.gphi, F)
            for d, s in faces:
                key, okey = (e, d, s), (self._nb(e, d, s), d, -s)
                n = np.broadcast_to(s * self.nunit[d], tr[key].shape[:-1] + (3,))
                Fc = rusanov(tr[key], tr[okey], n, g)
                if ns:
                    fv = 0.5 * (viscous_flux(tr[key], gtr[key], g, self.mu, self.pr)
                                + viscous_flux(tr[okey], gtr[okey], g, self.mu, self.pr))
                    Fc = Fc - np.einsum("fn,fnk->fk", n, fv)
                res -= np.einsum("f,fi,fk->ik", self.wface * self.nmag[d],
                                 self.phi_face[(d, s)], Fc)
            out[e] = res / self.M[:, None]
        return out
