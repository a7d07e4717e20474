"""Orthonormal polynomial bases and their gradients (test infrastructure only).

They span the solution space of each element type, so the nodal basis
l_z^(u) of Section 2 (l_z(x_s) = delta_zs) is ``V(x) @ inv(V(x_u))``:

* hexahedron: Q_p, tensor products of orthonormal Legendre polynomials;
* prism: P_p(triangle) x P_p(line), Dubiner triangle basis x Legendre;
* tetrahedron: P_p, Dubiner (collapsed-coordinate) basis;
* triangle / quadrilateral: the 2D analogues, used for face Lagrange bases.

Formulas: Hesthaven & Warburton (2008), Sections 6.1 and 10.1.
Pins (tests/test_oracle_basis.py): orthonormality under exact quadrature;
gradients against central finite differences; exact differentiation of
monomials through the derived nodal operators.
"""
import numpy as np

from .polys import djacobi, jacobi


def _tri_collapse(r, s):
    denom = np.where(np.abs(1.0 - s) > 1e-14, 1.0 - s, 1.0)
    a = np.where(np.abs(1.0 - s) > 1e-14, 2.0 * (1.0 + r) / denom - 1.0, -1.0)
    return a, s


def _tet_collapse(r, s, t):
    st = -s - t
    a = np.where(np.abs(st) > 1e-14,
                 2.0 * (1.0 + r) / np.where(np.abs(st) > 1e-14, st, 1.0) - 1.0,
                 -1.0)
    b = np.where(np.abs(1.0 - t) > 1e-14,
                 2.0 * (1.0 + s) / np.where(np.abs(1.0 - t) > 1e-14,
                                            1.0 - t, 1.0) - 1.0,
                 -1.0)
    return a, b, t


def tri_modes(p):
    return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]


def tet_modes(p):
    return [(i, j, k) for i in range(p + 1) for j in range(p + 1 - i)
            for k in range(p + 1 - i - j)]


def tri_basis(p, rs):
    r, s = rs[:, 0], rs[:, 1]
    a, b = _tri_collapse(r, s)
    cols = [np.sqrt(2.0) * jacobi(a, 0, 0, i) * jacobi(b, 2 * i + 1, 0, j)
            * (1.0 - b) ** i for i, j in tri_modes(p)]
    return np.stack(cols, axis=1)


def tri_grad(p, rs):
    r, s = rs[:, 0], rs[:, 1]
    a, b = _tri_collapse(r, s)
    dr, ds = [], []
    for i, j in tri_modes(p):
        fa, dfa = jacobi(a, 0, 0, i), djacobi(a, 0, 0, i)
        gb, dgb = jacobi(b, 2 * i + 1, 0, j), djacobi(b, 2 * i + 1, 0, j)
        h = 0.5 * (1.0 - b)
        mr = dfa * gb
        ms = dfa * gb * 0.5 * (1.0 + a)
        if i > 0:
            mr = mr * h ** (i - 1)
            ms = ms * h ** (i - 1)
        tmp = dgb * h ** i
        if i > 0:
            tmp = tmp - 0.5 * i * gb * h ** (i - 1)
        ms = ms + fa * tmp
        sc = 2.0 ** (i + 0.5)
        dr.append(mr * sc)
        ds.append(ms * sc)
    return np.stack(dr, axis=1), np.stack(ds, axis=1)


def tet_basis(p, x):
    a, b, c = _tet_collapse(x[:, 0], x[:, 1], x[:, 2])
    cols = []
    for i, j, k in tet_modes(p):
        cols.append(2.0 * np.sqrt(2.0) * jacobi(a, 0, 0, i)
                    * jacobi(b, 2 * i + 1, 0, j) * (1.0 - b) ** i
                    * jacobi(c, 2 * (i + j) + 2, 0, k) * (1.0 - c) ** (i + j))
    return np.stack(cols, axis=1)


def tet_grad(p, x):
    a, b, c = _tet_collapse(x[:, 0], x[:, 1], x[:, 2])
    gr, gs, gt = [], [], []
    for i, j, k in tet_modes(p):
        fa, dfa = jacobi(a, 0, 0, i), djacobi(a, 0, 0, i)
        gb, dgb = jacobi(b, 2 * i + 1, 0, j), djacobi(b, 2 * i + 1, 0, j)
        hc = jacobi(c, 2 * (i + j) + 2, 0, k)
        dhc = djacobi(c, 2 * (i + j) + 2, 0, k)
        hb = 0.5 * (1.0 - b)
        hcc = 0.5 * (1.0 - c)
        vr = dfa * gb * hc
        if i > 0:
            vr = vr * hb ** (i - 1)
        if i + j > 0:
            vr = vr * hcc ** (i + j - 1)
        vs = 0.5 * (1.0 + a) * vr
        tmp = dgb * hb ** i
        if i > 0:
            tmp = tmp - 0.5 * i * gb * hb ** (i - 1)
        if i + j > 0:
            tmp = tmp * hcc ** (i + j - 1)
        tmp = fa * tmp * hc
        vs = vs + tmp
        vt = 0.5 * (1.0 + a) * vr + 0.5 * (1.0 + b) * tmp
        tmp = dhc * hcc ** (i + j)
        if i + j > 0:
            tmp = tmp - 0.5 * (i + j) * hc * hcc ** (i + j - 1)
        tmp = fa * gb * tmp * hb ** i
        vt = vt + tmp
        sc = 2.0 ** (2 * i + j + 1.5)
        gr.append(vr * sc)
        gs.append(vs * sc)
        gt.append(vt * sc)
    return (np.stack(gr, axis=1), np.stack(gs, axis=1),
            np.stack(gt, axis=1))


def line_basis(p, x):
    return np.stack([jacobi(x, 0, 0, i) for i in range(p + 1)], axis=1)


def line_grad(p, x):
    return np.stack([djacobi(x, 0, 0, i) for i in range(p + 1)], axis=1)


def quad_basis(p, x):
    bx, by = line_basis(p, x[:, 0]), line_basis(p, x[:, 1])
    return np.stack([bx[:, i] * by[:, j]
                     for j in range(p + 1) for i in range(p + 1)], axis=1)


def hex_modes(p):
    return [(i, j, k) for k in range(p + 1) for j in range(p + 1)
            for i in range(p + 1)]


def hex_basis(p, x):
    b = [line_basis(p, x[:, d]) for d in range(3)]
    return np.stack([b[0][:, i] * b[1][:, j] * b[2][:, k]
                     for i, j, k in hex_modes(p)], axis=1)


def hex_grad(p, x):
    b = [line_basis(p, x[:, d]) for d in range(3)]
    g = [line_grad(p, x[:, d]) for d in range(3)]
    out = []
    for d in range(3):
        cols = []
        for idx in hex_modes(p):
            v = np.ones(len(x))
            for e in range(3):
                v = v * (g[e][:, idx[e]] if e == d else b[e][:, idx[e]])
            cols.append(v)
        out.append(np.stack(cols, axis=1))
    return tuple(out)


def pri_modes(p):
    return [(ij, k) for k in range(p + 1) for ij in tri_modes(p)]


def pri_basis(p, x):
    bt = tri_basis(p, x[:, :2])
    bl = line_basis(p, x[:, 2])
    nt = bt.shape[1]
    return np.stack([bt[:, m] * bl[:, k] for k in range(p + 1)
                     for m in range(nt)], axis=1)


def pri_grad(p, x):
    bt = tri_basis(p, x[:, :2])
    gr, gs = tri_grad(p, x[:, :2])
    bl = line_basis(p, x[:, 2])
    gl = line_grad(p, x[:, 2])
    nt = bt.shape[1]
    cols = [(gr[:, m] * bl[:, k], gs[:, m] * bl[:, k], bt[:, m] * gl[:, k])
            for k in range(p + 1) for m in range(nt)]
    return tuple(np.stack([c[d] for c in cols], axis=1) for d in range(3))

