"""Reference-element point sets for the oracle (test infrastructure only).

Section 2 places solution points x_z^(u) in the reference element and flux
points x_s^(f) on its surface, conforming across interfaces; Fig. 1 shows the
p=4 alpha-optimised tetrahedron sets and prints their coordinates.

* hexahedron: tensor Gauss-Legendre (GL) solution points; GL x GL flux points
  on each quadrilateral face (same 1D family).
* tetrahedron: warp-and-blend alpha-optimised nodes (Hesthaven & Warburton,
  Nodal DG Methods, 2008) with the book's 3D alpha table.
* triangle faces: the warp-and-blend triangle evaluated with the *3D* alpha of
  the same order.  This is the face restriction of the tetrahedron set, so the
  tetrahedron's flux points are a subset of its solution points as Fig. 1(b,c)
  show.  Pinned: the p=4 coordinates printed in Fig. 1 (-0.551583572090994,
  0.103167144181987, +-0.654653670707977, centroid -0.5) are reproduced to
  15 digits by tests/test_oracle_points.py.
* prism: warp-and-blend triangle with the book's 2D alpha table, tensored
  with GL points along the prism axis (reading; parity unpinned except by
  construction and symmetry).

Reference elements: hex [-1,1]^3; prism = triangle {(-1,-1),(1,-1),(-1,1)}
x [-1,1]; tet with vertices (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1).
"""
import numpy as np

from .polys import gauss_legendre, gauss_lobatto, jacobi

ALPHA_2D = [0.0, 0.0, 1.4152, 0.1001, 0.2751, 0.9800, 1.0999, 1.2832,
            1.3648, 1.4773, 1.4959, 1.5743, 1.5770, 1.6223, 1.6258]
ALPHA_3D = [0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577, 1.1603,
            1.10153, 0.6080, 0.4523, 0.8856, 0.8717, 0.9655]


def _warp(n, r):
    """1D warp: GLL minus equispaced, interpolated and divided by 1 - r^2."""
    lgl, _ = gauss_lobatto(n + 1)
    req = np.linspace(-1.0, 1.0, n + 1)
    veq = np.array([jacobi(req, 0, 0, i) for i in range(n + 1)]).T
    pm = np.array([jacobi(r, 0, 0, i) for i in range(n + 1)])
    lm = np.linalg.solve(veq.T, pm)
    warp = lm.T @ (lgl - req)
    inside = np.abs(r) < 1.0 - 1e-10
    sf = 1.0 - (inside * r) ** 2
    return warp / sf + warp * (inside - 1.0)


def _tri_shift(n, alpha, l1, l2, l3):
    """Warp-and-blend displacement on the equilateral triangle."""
    w1 = _warp(n, l3 - l2)
    w2 = _warp(n, l1 - l3)
    w3 = _warp(n, l2 - l1)
    f1 = 4 * l2 * l3 * w1 * (1 + (alpha * l1) ** 2)
    f2 = 4 * l1 * l3 * w2 * (1 + (alpha * l2) ** 2)
    f3 = 4 * l1 * l2 * w3 * (1 + (alpha * l3) ** 2)
    c2, s2 = np.cos(2 * np.pi / 3), np.sin(2 * np.pi / 3)
    c4, s4 = np.cos(4 * np.pi / 3), np.sin(4 * np.pi / 3)
    return f1 + c2 * f2 + c4 * f3, s2 * f2 + s4 * f3


def tri_nodes(n, alpha):
    """Warp-and-blend nodes on the reference triangle, order n, as (N, 2)."""
    l1, l3 = [], []
    for i in range(n + 1):
        for j in range(n + 1 - i):
            l1.append(i / n)
            l3.append(j / n)
    l1 = np.array(l1)
    l3 = np.array(l3)
    l2 = 1.0 - l1 - l3
    x = -l2 + l3
    y = (-l2 - l3 + 2 * l1) / np.sqrt(3.0)
    dx, dy = _tri_shift(n, alpha, l1, l2, l3)
    x = x + dx
    y = y + dy
    # equilateral -> reference triangle through barycentric coordinates
    b1 = (np.sqrt(3.0) * y + 1.0) / 3.0
    b2 = (-3.0 * x - np.sqrt(3.0) * y + 2.0) / 6.0
    b3 = (3.0 * x - np.sqrt(3.0) * y + 2.0) / 6.0
    r = -b2 + b3 - b1
    s = -b2 - b3 + b1
    return np.stack([r, s], axis=1)


def _evalwarp(n, xnodes, xout):
    xeq = np.array([-1.0 + 2.0 * (n - i) / n for i in range(n + 1)])
    warp = np.zeros_like(xout)
    for i in range(n + 1):
        d = np.full_like(xout, xnodes[i] - xeq[i])
        for j in range(1, n):
            if i != j:
                d = d * (xout - xeq[j]) / (xeq[i] - xeq[j])
        if i != 0:
            d = -d / (xeq[i] - xeq[0])
        if i != n:
            d = d / (xeq[i] - xeq[n])
        warp = warp + d
    return warp


def _evalshift(n, alpha, l1, l2, l3):
    gx = -gauss_lobatto(n + 1)[0]
    w1 = _evalwarp(n, gx, l3 - l2)
    w2 = _evalwarp(n, gx, l1 - l3)
    w3 = _evalwarp(n, gx, l2 - l1)
    f1 = 4 * l2 * l3 * w1 * (1 + (alpha * l1) ** 2)
    f2 = 4 * l3 * l1 * w2 * (1 + (alpha * l2) ** 2)
    f3 = 4 * l1 * l2 * w3 * (1 + (alpha * l3) ** 2)
    c2, s2 = np.cos(2 * np.pi / 3), np.sin(2 * np.pi / 3)
    c4, s4 = np.cos(4 * np.pi / 3), np.sin(4 * np.pi / 3)
    return f1 + c2 * f2 + c4 * f3, s2 * f2 + s4 * f3


def tet_nodes(n):
    """Alpha-optimised warp-and-blend nodes on the reference tet, (N, 3)."""
    alpha = ALPHA_3D[n - 1] if n <= 15 else 1.0
    r, s, t = [], [], []
    for k in range(n + 1):
        for j in range(n + 1 - k):
            for i in range(n + 1 - k - j):
                r.append(-1.0 + 2.0 * i / n)
                s.append(-1.0 + 2.0 * j / n)
                t.append(-1.0 + 2.0 * k / n)
    r, s, t = np.array(r), np.array(s), np.array(t)
    L1 = (1 + t) / 2
    L2 = (1 + s) / 2
    L3 = -(1 + r + s + t) / 2
    L4 = (1 + r) / 2
    v1 = np.array([-1.0, -1.0 / np.sqrt(3), -1.0 / np.sqrt(6)])
    v2 = np.array([1.0, -1.0 / np.sqrt(3), -1.0 / np.sqrt(6)])
    v3 = np.array([0.0, 2.0 / np.sqrt(3), -1.0 / np.sqrt(6)])
    v4 = np.array([0.0, 0.0, 3.0 / np.sqrt(6)])
    t1 = [v2 - v1, v2 - v1, v3 - v2, v3 - v1]
    t2 = [v3 - 0.5 * (v1 + v2), v4 - 0.5 * (v1 + v2),
          v4 - 0.5 * (v2 + v3), v4 - 0.5 * (v1 + v3)]
    t1 = [v / np.linalg.norm(v) for v in t1]
    t2 = [v / np.linalg.norm(v) for v in t2]
    xyz = (np.outer(L3, v1) + np.outer(L4, v2) + np.outer(L2, v3)
           + np.outer(L1, v4))
    shift = np.zeros_like(xyz)
    tol = 1e-10
    faces = [(L1, L2, L3, L4), (L2, L1, L3, L4),
             (L3, L1, L4, L2), (L4, L1, L3, L2)]
    for f, (La, Lb, Lc, Ld) in enumerate(faces):
        w1, w2 = _evalshift(n, alpha, Lb, Lc, Ld)
        blend = Lb * Lc * Ld
        denom = (Lb + 0.5 * La) * (Lc + 0.5 * La) * (Ld + 0.5 * La)
        ok = denom > tol
        blend = np.where(ok, (1 + (alpha * La) ** 2) * blend
                         / np.where(ok, denom, 1.0), blend)
        shift += np.outer(blend * w1, t1[f]) + np.outer(blend * w2, t2[f])
        edge = (La < tol) & (((Lb > tol).astype(int) + (Lc > tol)
                              + (Ld > tol)) < 3)
        shift[edge] = (np.outer(w1[edge], t1[f])
                       + np.outer(w2[edge], t2[f]))
    xyz = xyz + shift
    # equilateral tet -> reference tet through barycentric coordinates
    A = np.stack([v2 - v1, v3 - v1, v4 - v1], axis=1)
    lam = np.linalg.solve(A, (xyz - v1).T).T   # weights of v2, v3, v4
    return -1.0 + 2.0 * lam


def tri_face_points(p):
    """Flux points of a triangular face (restriction of the tet set)."""
    if p == 0:
        return np.array([[-1.0 / 3.0, -1.0 / 3.0]])
    return tri_nodes(p, ALPHA_3D[p - 1] if p <= 15 else 1.0)


def tri_solution_points(p):
    """Alpha-optimised (2D table) warp-and-blend triangle nodes."""
    if p == 0:
        return np.array([[-1.0 / 3.0, -1.0 / 3.0]])
    return tri_nodes(p, ALPHA_2D[p - 1] if p <= 15 else 5.0 / 3.0)


def gl_points(p):
    return gauss_legendre(p + 1)[0]
