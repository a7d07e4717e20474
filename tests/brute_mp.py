"""Brute-force FR right-hand side at 50 significant digits (test
infrastructure; imports nothing from ``oracle/`` or the library).

It restates the definitions of the paper's Section 2 for hexahedra with an
affine map, one scalar at a time in mpmath:

* solution points: the N = p + 1 roots of the Legendre polynomial P_N (Newton
  iteration on the three-term recurrence), or the N Gauss-Lobatto points
  (+-1 and the roots of P'_p), tensorised; flux points: the same 1D points
  on each face;
* Lagrange basis l_m and its derivative from the product formula;
* Eq. (disu): traces by Lagrange interpolation along the line through the
  face point;
* Eq. (comm_flux): Rusanov, F = (F(u-) + F(u+)).n / 2 - lambda (u+ - u-) / 2
  with lambda = max(|v- . n| + c-, |v+ . n| + c+), n the physical unit normal;
* Eq. (FRfinal) with the DG correction function written by formula: the right
  Radau polynomial g_R = (P_{p+1} + P_p) / 2 (Huynh 2007), so the correction of
  a plus face at line position x is g_R'(x) and of a minus face g_R'(-x);
* du/dt = -(1/det J) div~ f~ with f~ = det J J^{-1} f;
* Navier-Stokes (BR1): u^C = (u- + u+)/2, corrected reference gradient,
  physical gradient J^{-T} grad~ u, viscous flux in primitive variables
  (stress mu (grad v + grad v^T - 2/3 div v I), heat flux kappa grad e with
  e = p / ((gamma - 1) rho) and kappa = mu gamma / Pr), viscous common flux
  the average of both sides'.

Mesh: an nx x ny x nz block of parallelepipeds, element (i, j, k) being the
image of [2i, 2i+2] x [2j, 2j+2] x [2k, 2k+2] under x = A xi, periodic in all
three directions with translations A (2nx, 0, 0), A (0, 2ny, 0),
A (0, 0, 2nz).
"""
import itertools

import mpmath as mp
import numpy as np


def _legendre(n, x):
    """(P_n(x), P_n'(x)) by the three-term recurrence."""
    p0, p1 = mp.mpf(1), x
    if n == 0:
        return p0, mp.mpf(0)
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # P_n' = n (x P_n - P_{n-1}) / (x^2 - 1), valid inside (-1, 1); at the
    # end points P_n'(+-1) = (+-1)^{n-1} n (n + 1) / 2
    if abs(x) == 1:
        d = mp.mpf(n * (n + 1)) / 2 * (x ** (n - 1))
    else:
        d = n * (x * p1 - p0) / (x * x - 1)
    return p1, d


def gauss_points(n):
    pts = []
    for i in range(n):
        x = mp.cos(mp.pi * (i + mp.mpf(3) / 4) / (n + mp.mpf(1) / 2))
        for _ in range(200):
            pv, dv = _legendre(n, x)
            dx = pv / dv
            x -= dx
            if abs(dx) < mp.mpf(10) ** (-mp.mp.dps + 2):
                break
        pts.append(x)
    return sorted(pts)


def lobatto_points(n):
    """The n Gauss-Lobatto points: +-1 and the roots of P'_{n-1} (Newton,
    with P'' from Legendre's equation (1 - x^2) P'' = 2 x P' - m(m+1) P)."""
    m = n - 1
    inner = []
    for i in range(1, m):
        x = -mp.cos(mp.pi * i / m)
        for _ in range(200):
            pv, dv = _legendre(m, x)
            d2 = (2 * x * dv - m * (m + 1) * pv) / (1 - x * x)
            dx = dv / d2
            x -= dx
            if abs(dx) < mp.mpf(10) ** (-mp.mp.dps + 2):
                break
        inner.append(x)
    return [mp.mpf(-1)] + sorted(inner) + [mp.mpf(1)]


def lagrange(xs, j, x):
    v = mp.mpf(1)
    for m, xm in enumerate(xs):
        if m != j:
            v *= (x - xm) / (xs[j] - xm)
    return v


def dlagrange(xs, j, x):
    tot = mp.mpf(0)
    for m, xm in enumerate(xs):
        if m == j:
            continue
        t = 1 / (xs[j] - xm)
        for k, xk in enumerate(xs):
            if k != j and k != m:
                t *= (x - xk) / (xs[j] - xk)
        tot += t
    return tot


def radau_right_slope(p, x):
    """g_R'(x) of the DG correction function g_R = (P_{p+1} + P_p)/2."""
    return (_legendre(p + 1, x)[1] + _legendre(p, x)[1]) / 2


def _mat_inv_t(A):
    M = mp.matrix(A)
    return M ** -1, mp.det(M)


class BruteFR:
    def __init__(self, p, A, n, gamma=1.4, mu=0.0, pr=0.72, dps=50, family="gl"):
        mp.mp.dps = dps
        self.p, self.N = p, p + 1
        self.n = tuple(n)
        self.A = mp.matrix([[mp.mpf(float(a)) for a in row] for row in A])
        self.Ainv, self.det = _mat_inv_t(self.A)
        self.gamma, self.mu, self.pr = mp.mpf(gamma), mp.mpf(mu), mp.mpf(pr)
        self.x1 = lobatto_points(self.N) if family == "gll" else gauss_points(self.N)
        N = self.N
        self.lm = [lagrange(self.x1, m, mp.mpf(-1)) for m in range(N)]
        self.lp = [lagrange(self.x1, m, mp.mpf(1)) for m in range(N)]
        self.dl = [[dlagrange(self.x1, m, self.x1[a]) for m in range(N)]
                   for a in range(N)]
        self.gp = [radau_right_slope(p, self.x1[a]) for a in range(N)]
        self.gm = [radau_right_slope(p, -self.x1[a]) for a in range(N)]
        self.elems = list(itertools.product(range(n[0]), range(n[1]), range(n[2])))
        # physical normal vector det J J^{-T} e_d of a plus face in direction d
        self.nvec = [[self.det * self.Ainv[d, k] for k in range(3)]
                     for d in range(3)]
        self.nmag = [mp.sqrt(sum(c * c for c in v)) for v in self.nvec]

    # ---------------------------------------------------------------- geometry
    def point(self, e, abc):
        xi = [self.x1[abc[d]] + 2 * e[d] + 1 for d in range(3)]
        return [sum(self.A[k, d] * xi[d] for d in range(3)) for k in range(3)]

    def points(self):
        """Float positions of every solution point, keyed (elem, a, b, c)."""
        out = {}
        N = self.N
        for e in self.elems:
            for abc in itertools.product(range(N), repeat=3):
                out[(e,) + abc] = [float(v) for v in self.point(e, abc)]
        return out

    def neighbour(self, e, d, s):
        f = list(e)
        f[d] = (f[d] + s) % self.n[d]
        return tuple(f)

    @staticmethod
    def line(d, i, j, m):
        if d == 0:
            return (m, i, j)
        if d == 1:
            return (i, m, j)
        return (i, j, m)

    # ---------------------------------------------------------------- physics
    def prim(self, u):
        rho = u[0]
        v = [u[1] / rho, u[2] / rho, u[3] / rho]
        p = (self.gamma - 1) * (u[4] - rho * sum(c * c for c in v) / 2)
        return rho, v, p

    def euler(self, u):
        rho, v, p = self.prim(u)
        F = []
        for j in range(3):
            row = [u[1 + j]] + [u[1 + i] * v[j] + (p if i == j else 0)
                                for i in range(3)] + [(u[4] + p) * v[j]]
            F.append(row)
        return F

    def viscous(self, u, g):
        """g[n][k] = d u_k / d x_n.  Primitive form of the viscous flux."""
        gm1 = self.gamma - 1
        rho, v, p = self.prim(u)
        grho = [g[n][0] for n in range(3)]
        # d v_i / d x_n from the quotient rule on rho v_i
        gv = [[(g[n][1 + i] - v[i] * grho[n]) / rho for i in range(3)]
              for n in range(3)]
        # pressure gradient: p = (gamma-1)(E - |m|^2 / (2 rho))
        gp = [gm1 * (g[n][4] - sum(v[i] * g[n][1 + i] for i in range(3))
                     + sum(c * c for c in v) / 2 * grho[n]) for n in range(3)]
        # e = p / ((gamma - 1) rho)
        ge = [(gp[n] - p * grho[n] / rho) / (gm1 * rho) for n in range(3)]
        div = gv[0][0] + gv[1][1] + gv[2][2]
        kappa = self.mu * self.gamma / self.pr
        F = []
        for n in range(3):
            tau = [self.mu * (gv[n][i] + gv[i][n]) - (2 * self.mu * div / 3 if i == n else 0)
                   for i in range(3)]
            F.append([mp.mpf(0)] + tau
                     + [sum(v[i] * tau[i] for i in range(3)) + kappa * ge[n]])
        return F

    def rusanov(self, ul, ur, n):
        fl, fr = self.euler(ul), self.euler(ur)
        rl, vl, pl = self.prim(ul)
        rr, vr, pr_ = self.prim(ur)
        cl = mp.sqrt(self.gamma * pl / rl)
        cr = mp.sqrt(self.gamma * pr_ / rr)
        lam = max(abs(sum(vl[k] * n[k] for k in range(3))) + cl,
                  abs(sum(vr[k] * n[k] for k in range(3))) + cr)
        return [sum((fl[j][k] + fr[j][k]) * n[j] for j in range(3)) / 2
                - lam * (ur[k] - ul[k]) / 2 for k in range(5)]

    # ---------------------------------------------------------------- RHS
    def _trace(self, field, e, d, s, i, j):
        """Value of a per-point list field at face (d, s) point (i, j)."""
        w = self.lp if s > 0 else self.lm
        first = field[(e,) + self.line(d, i, j, 0)]
        out = [mp.mpf(0)] * len(first)
        for m in range(self.N):
            f = field[(e,) + self.line(d, i, j, m)]
            for k in range(len(out)):
                out[k] += w[m] * f[k]
        return out

    def _faces(self):
        N = self.N
        for e in self.elems:
            for d in range(3):
                for s in (-1, 1):
                    for i in range(N):
                        for j in range(N):
                            yield e, d, s, i, j

    def rhs(self, u_np, physics="euler"):
        """u_np: {(elem, a, b, c): 5 floats}.  Returns the same keys -> 5 mpf."""
        N = self.N
        ns = physics == "ns"
        u = {k: [mp.mpf(float(c)) for c in v] for k, v in u_np.items()}
        unit = [[c / self.nmag[d] for c in self.nvec[d]] for d in range(3)]
        # traces on every face point (own side)
        tr = {f: self._trace(u, *f) for f in self._faces()}

        def other(e, d, s, i, j):
            return tr[(self.neighbour(e, d, s), d, -s, i, j)]

        grad = None
        if ns:
            uc = {f: [(a + b) / 2 for a, b in zip(tr[f], other(*f))]
                  for f in tr}
            grad = {}
            for e in self.elems:
                for abc in itertools.product(range(N), repeat=3):
                    gref = []
                    for d in range(3):
                        a = abc[d]
                        i, j = [abc[q] for q in range(3) if q != d]
                        val = [mp.mpf(0)] * 5
                        for m in range(N):
                            um = u[(e,) + self.line(d, i, j, m)]
                            for k in range(5):
                                val[k] += self.dl[a][m] * um[k]
                        for s, w in ((1, self.gp[a]), (-1, self.gm[a])):
                            f = (e, d, s, i, j)
                            for k in range(5):
                                val[k] += w * s * (uc[f][k] - tr[f][k])
                        gref.append(val)
                    grad[(e,) + abc] = [[sum(self.Ainv[d, n] * gref[d][k]
                                             for d in range(3))
                                         for k in range(5)] for n in range(3)]
            gflat = {k: [c for row in v for c in row] for k, v in grad.items()}
            gtr = {f: self._trace(gflat, *f) for f in self._faces()}

            def g3(flat):
                return [flat[5 * n:5 * n + 5] for n in range(3)]

        # transformed flux at solution points
        ft = {}
        for key, uz in u.items():
            F = self.euler(uz)
            if ns:
                Fv = self.viscous(uz, grad[key])
                F = [[F[n][k] - Fv[n][k] for k in range(5)] for n in range(3)]
            ft[key] = [[self.det * sum(self.Ainv[d, n] * F[n][k] for n in range(3))
                        for k in range(5)] for d in range(3)]
        out = {}
        for e in self.elems:
            for abc in itertools.product(range(N), repeat=3):
                div = [mp.mpf(0)] * 5
                for d in range(3):
                    a = abc[d]
                    i, j = [abc[q] for q in range(3) if q != d]
                    for m in range(N):
                        fm = ft[(e,) + self.line(d, i, j, m)][d]
                        for k in range(5):
                            div[k] += self.dl[a][m] * fm[k]
                    for s, w in ((1, self.gp[a]), (-1, self.gm[a])):
                        f = (e, d, s, i, j)
                        n = [s * c for c in unit[d]]
                        ul, ur = tr[f], other(*f)
                        F = self.rusanov(ul, ur, n)
                        if ns:
                            gl = g3(gtr[f])
                            gr = g3(gtr[(self.neighbour(e, d, s), d, -s, i, j)])
                            Fl, Fr = self.viscous(ul, gl), self.viscous(ur, gr)
                            F = [F[k] - sum((Fl[q][k] + Fr[q][k]) * n[q]
                                            for q in range(3)) / 2
                                 for k in range(5)]
                        # own transformed normal flux at the face point
                        fn = [mp.mpf(0)] * 5
                        wt = self.lp if s > 0 else self.lm
                        for m in range(N):
                            fm = ft[(e,) + self.line(d, i, j, m)][d]
                            for k in range(5):
                                fn[k] += s * wt[m] * fm[k]
                        for k in range(5):
                            div[k] += w * (self.nmag[d] * F[k] - fn[k])
                out[(e,) + abc] = [-c / self.det for c in div]
        return out


def spec_for(A, n):
    """Mesh description (library / oracle input format) of the block."""
    A = np.asarray(A, float)
    nx, ny, nz = n
    lat = [np.arange(0, 2 * k + 1, 2, dtype=float) for k in n]

    def nid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    xi = np.array([[lat[0][i], lat[1][j], lat[2][k]]
                   for k in range(nz + 1) for j in range(ny + 1)
                   for i in range(nx + 1)])
    nodes = xi @ A.T
    conn = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                conn.append([nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k),
                             nid(i, j + 1, k), nid(i, j, k + 1), nid(i + 1, j, k + 1),
                             nid(i + 1, j + 1, k + 1), nid(i, j + 1, k + 1)])
    periodic = [A @ np.array([2.0 * nx, 0, 0]), A @ np.array([0, 2.0 * ny, 0]),
                A @ np.array([0, 0, 2.0 * nz])]
    return {"nodes": nodes, "elements": {"hex": np.array(conn, np.int64)},
            "periodic": [list(v) for v in periodic], "bfaces": [], "maps": {}}


def random_state(keys, seed, amp=0.3, gamma=1.4):
    """Discontinuous random conserved state at every solution point: rho and
    p uniform in [1 - amp, 1 + amp], velocity components in [-amp, amp]
    (a small amp keeps the extrapolated face traces positive at high p)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for k in sorted(keys):
        rho = rng.uniform(1 - amp, 1 + amp)
        v = rng.uniform(-amp, amp, 3)
        p = rng.uniform(1 - amp, 1 + amp)
        out[k] = np.array([rho, *(rho * v), p / (gamma - 1) + 0.5 * rho * v @ v])
    return out
