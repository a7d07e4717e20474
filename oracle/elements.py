"""Reference element types and their FR operators (test infrastructure only).

For each element type this builds, in FP64, from the definitions of
Section 2 of the paper:

* the vertex map x = M_n(x~) (trilinear hex, linear prism, affine tet) and
  its derivatives, for the Jacobian J = dM/dx~ of Section 2;
* solution points, flux points on every face, reference unit outward
  normals at the flux points and each face's area scale; hexahedra take
  Gauss-Legendre (default) or Gauss-Lobatto line points (``family``);
* ``M0[s, z] = l_z(x_s^(f))``  -- Eq. (disu), interpolation to flux points;
* ``D[d][z, v] = d l_v / d x~_d (x_z)`` -- the grad l term of Eq. (FRfinal);
* ``LIFT[z, s] = (div~ g_s)(x_z)`` -- the correction term of Eq. (FRfinal).
  The paper names only "a flux correction function g".  Reading: the DG
  choice (Huynh 2007).  For every type it is the DG lift: div~ g_s lies in
  the solution space and satisfies, for every v in that space,
  int_element v div~ g_s = int_face(s) v l_s^(f), where l_s^(f) is the face
  Lagrange basis of the flux points.  Face integrals use exact Gauss rules.
  Pin: on the hexahedron it equals the tensor-product right/left Radau form
  g_R' = (P'_{p+1} + P'_p)/2 (tests/test_oracle_operators.py).
* integration weights ``W[z] = int l_z`` for discrete conservation checks.
* anti-aliasing (Section 3.2, "Anti-aliasing"): a volume quadrature rule of
  degree qdeg, ``B[q, z] = l_z(x_q)`` (solution -> quadrature points) and the
  least-squares projection ``P[z, q]`` onto the solution space: with the
  orthonormal basis phi_k, the projection of f has modal coefficients
  c_k = sum_q w_q phi_k(x_q) f(x_q), so P = V Phi_q^T diag(w).  Reading: the
  paper's Polyquad rules are not available here; the rules are collapsed
  Gauss-Jacobi products (tensor Gauss on the hexahedron), exact to degree
  2n - 1 with n = qdeg // 2 + 1 points per direction.
"""
import numpy as np

from . import bases
from .points import gl_points, tet_nodes, tri_face_points, tri_solution_points
from .polys import gauss_jacobi, gauss_legendre, gauss_lobatto

SQ2 = np.sqrt(2.0)
SQ3 = np.sqrt(3.0)


def _quad_rule(n):
    x, w = gauss_legendre(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    W = np.outer(w, w)
    return np.stack([X.ravel(), Y.ravel()], axis=1), W.ravel()


def _tri_rule(n):
    a, wa = gauss_legendre(n)
    b, wb = gauss_jacobi(n, 1.0, 0.0)
    A, B = np.meshgrid(a, b, indexing="ij")
    r = 0.5 * (1 + A) * (1 - B) - 1
    s = B
    w = np.outer(wa, wb) / 2.0
    return np.stack([r.ravel(), s.ravel()], axis=1), w.ravel()


def tet_rule(n):
    a, wa = gauss_legendre(n)
    b, wb = gauss_jacobi(n, 1.0, 0.0)
    c, wc = gauss_jacobi(n, 2.0, 0.0)
    A, B, C = np.meshgrid(a, b, c, indexing="ij")
    r = 0.25 * (1 + A) * (1 - B) * (1 - C) - 1
    s = 0.5 * (1 + B) * (1 - C) - 1
    w = (wa[:, None, None] * wb[None, :, None] * wc[None, None, :]) / 8.0
    return np.stack([r.ravel(), s.ravel(), C.ravel()], axis=1), w.ravel()


def hex_rule(n):
    x, w = gauss_legendre(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), W.ravel()


def pri_rule(n):
    t2, w2 = _tri_rule(n)
    z, wz = gauss_legendre(n)
    pts = np.concatenate([np.column_stack([t2, np.full(len(t2), zz)])
                          for zz in z])
    w = np.concatenate([w2 * wzz for wzz in wz])
    return pts, w


def _cubic_simplex(lam, dlam, edges, faces):
    """Cubic Lagrange basis on a simplex (a triangle or a tetrahedron) from
    its barycentric coordinates lam (npts, n_vertices), whose gradients
    dlam[v] are constant.  Nodes, in this order: the vertices; two per edge
    (a, b), at barycentric (2/3, 1/3) then (1/3, 2/3) of its two vertices;
    the centroid of each face (a, b, c).  Basis: 9/2 l (l - 1/3)(l - 2/3)
    at a vertex, 27/2 l_a l_b (l_a - 1/3) at an edge node nearer a,
    27 l_a l_b l_c at a face centroid.  Returns the values (npts, n) and the
    derivatives (ndim, npts, n)."""
    ndim = len(dlam[0])
    vals, ders = [], [[] for _ in range(ndim)]

    def push(v, grad_by_vertex):
        vals.append(v)
        for j in range(ndim):
            ders[j].append(sum(g * dlam[w][j] for w, g in grad_by_vertex))

    for v in range(lam.shape[1]):
        lv = lam[:, v]
        push(0.5 * lv * (3 * lv - 1) * (3 * lv - 2),
             [(v, 0.5 * (27 * lv * lv - 18 * lv + 2))])
    for a, b in edges:
        for s, t in ((a, b), (b, a)):
            ls, lt = lam[:, s], lam[:, t]
            push(4.5 * ls * lt * (3 * ls - 1),
                 [(s, 4.5 * lt * (6 * ls - 1)), (t, 4.5 * ls * (3 * ls - 1))])
    for a, b, c in faces:
        la, lb, lc = lam[:, a], lam[:, b], lam[:, c]
        push(27 * la * lb * lc, [(a, 27 * lb * lc), (b, 27 * la * lc), (c, 27 * la * lb)])
    return np.stack(vals, axis=1), np.stack([np.stack(d, axis=1) for d in ders])


def _cubic_simplex_nodes(verts, edges, faces):
    """Reference coordinates of the nodes of _cubic_simplex."""
    v = np.asarray(verts, float)
    out = list(v)
    for a, b in edges:
        out += [(2 * v[a] + v[b]) / 3, (v[a] + 2 * v[b]) / 3]
    for f in faces:
        out.append(v[list(f)].mean(axis=0))
    return np.array(out)


class Face:
    """One face of a reference element: 2D parameterisation -> 3D."""

    def __init__(self, kind, verts, origin, ds, dt, normal):
        self.kind = kind            # 'quad' or 'tri'
        self.verts = verts          # local vertex ids
        self.origin = np.asarray(origin, float)
        self.ds = np.asarray(ds, float)   # d x~ / d s
        self.dt = np.asarray(dt, float)   # d x~ / d t
        self.normal = np.asarray(normal, float)
        self.scale = np.linalg.norm(np.cross(self.ds, self.dt))

    def map(self, st):
        return (self.origin[None, :] + st[:, :1] * self.ds[None, :]
                + st[:, 1:2] * self.dt[None, :])


class ElementType:
    """Base class: subclasses fill the geometry tables and bases."""

    name = None
    nverts = 0

    def __init__(self, p, family="gl"):
        self.p = p
        self.family = family
        self.upts = self.solution_points()
        self.nupts = len(self.upts)
        fp, fidx, fnrm = [], [], []
        self.face_fpts = []
        for fi, face in enumerate(self.faces):
            st = self.face_points(face)
            x = face.map(st)
            start = sum(len(a) for a in fp)
            fp.append(x)
            fidx += [fi] * len(x)
            fnrm.append(np.tile(face.normal, (len(x), 1)))
            self.face_fpts.append(np.arange(start, start + len(x)))
        self.fpts = np.concatenate(fp)
        self.fpts_face = np.array(fidx)
        self.fpts_norm = np.concatenate(fnrm)
        self.nfpts = len(self.fpts)
        self._build_operators()

    # face Lagrange basis and exact face quadrature ---------------------
    def line_points(self):
        """1D point set of the tensor-product directions: Gauss-Legendre, or
        Gauss-Lobatto for the hexahedron family "gll" (flux points are then
        solution points: Section 3.1, "Matrix multiplications")."""
        if self.family == "gll":
            return gauss_lobatto(self.p + 1)[0]
        return gl_points(self.p)

    def face_points(self, face):
        p = self.p
        if face.kind == "quad":
            x = self.line_points()
            X, Y = np.meshgrid(x, x, indexing="xy")
            return np.stack([X.ravel(), Y.ravel()], axis=1)
        return tri_face_points(p)

    def _face_basis(self, face, st):
        if face.kind == "quad":
            return bases.quad_basis(self.p, st)
        return bases.tri_basis(self.p, st)

    def _face_rule(self, face):
        n = self.p + 2
        return _quad_rule(n) if face.kind == "quad" else _tri_rule(n)

    def _build_operators(self):
        V = self.basis(self.upts)
        Vi = np.linalg.inv(V)
        self.vdm_inv = Vi
        self.M0 = self.basis(self.fpts) @ Vi
        G = self.grad(self.upts)
        self.D = [g @ Vi for g in G]
        # DG lift of every flux point (orthonormal basis => mass = I)
        lift = np.zeros((self.nupts, self.nfpts))
        for fi, face in enumerate(self.faces):
            st_q, w_q = self._face_rule(face)
            xq = face.map(st_q)
            psi_q = self.basis(xq)                           # (nq, nmodes)
            st_f = self.face_points(face)
            Vf = self._face_basis(face, st_f)
            lf = self._face_basis(face, st_q) @ np.linalg.inv(Vf)   # (nq, nf)
            b = psi_q.T @ (w_q[:, None] * face.scale * lf)   # (nmodes, nf)
            lift[:, self.face_fpts[fi]] = V @ b
        self.LIFT = lift
        # integration weights of the nodal basis
        xq, wq = self.volume_rule(self.p + 2)
        self.W = (self.basis(xq) @ Vi).T @ wq

    # anti-aliasing ---------------------------------------------------------
    def quadrature(self, qdeg):
        """Volume rule exact for polynomials of degree qdeg."""
        return self.volume_rule(qdeg // 2 + 1)

    def aa_operators(self, qdeg):
        """(xq, wq, B, P): quadrature points and weights, interpolation from
        the solution points, least-squares projection back onto them."""
        xq, wq = self.quadrature(qdeg)
        phi = self.basis(xq)                                 # (nq, nmodes)
        B = phi @ self.vdm_inv
        P = self.basis(self.upts) @ (phi.T * wq[None, :])
        return xq, wq, B, P

    # geometry of the vertex map ------------------------------------------
    def map_points(self, verts, x):
        """Physical coordinates of reference points x, verts (ne, nv, 3)."""
        N = self.shape(x)                                    # (npts, nv)
        return np.einsum("pv,evk->epk", N, verts)

    def jacobian(self, verts, x):
        """a[e, p, j, :] = d x / d x~_j at reference points x."""
        dN = self.dshape(x)                                  # (3, npts, nv)
        return np.einsum("jpv,evk->epjk", dN, verts)

    def metrics(self, verts, x):
        """Return (S, detJ): S = detJ * J^{-1}, f~ = S f, rows a_j x a_k."""
        a = self.jacobian(verts, x)
        S = np.stack([np.cross(a[:, :, 1], a[:, :, 2]),
                      np.cross(a[:, :, 2], a[:, :, 0]),
                      np.cross(a[:, :, 0], a[:, :, 1])], axis=2)
        det = np.einsum("epk,epk->ep", a[:, :, 0], S[:, :, 0])
        return S, det


class Hex(ElementType):
    name = "hex"
    nverts = 8
    signs = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                      [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float)
    faces = [
        Face("quad", (0, 3, 7, 4), (-1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0)),
        Face("quad", (1, 2, 6, 5), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 0)),
        Face("quad", (0, 1, 5, 4), (0, -1, 0), (1, 0, 0), (0, 0, 1), (0, -1, 0)),
        Face("quad", (3, 2, 6, 7), (0, 1, 0), (1, 0, 0), (0, 0, 1), (0, 1, 0)),
        Face("quad", (0, 1, 2, 3), (0, 0, -1), (1, 0, 0), (0, 1, 0), (0, 0, -1)),
        Face("quad", (4, 5, 6, 7), (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ]

    def solution_points(self):
        x = self.line_points()
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def basis(self, x):
        return bases.hex_basis(self.p, x)

    def grad(self, x):
        return bases.hex_grad(self.p, x)

    def volume_rule(self, n):
        return hex_rule(n)

    def shape(self, x):
        s = self.signs
        return np.prod(1 + x[:, None, :] * s[None, :, :], axis=2) / 8.0

    def dshape(self, x):
        s = self.signs
        f = 1 + x[:, None, :] * s[None, :, :]            # (npts, 8, 3)
        out = []
        for j in range(3):
            d = s[None, :, j] / 8.0
            for k in range(3):
                if k != j:
                    d = d * f[:, :, k]
            out.append(d)
        return np.stack(out)


    # quadratic map (27 nodes, tensor order a + 3b + 9c at (-1+a, -1+b, -1+c))
    def q2_nodes(self):
        a = np.array([-1.0, 0.0, 1.0])
        c, b, aa = np.meshgrid(a, a, a, indexing="ij")
        return np.stack([aa.ravel(), b.ravel(), c.ravel()], axis=1)

    def curl_nodes(self):
        g = gauss_lobatto(self.p + 1)[0]
        c, b, a = np.meshgrid(g, g, g, indexing="ij")
        return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)

    @staticmethod
    def _lag2(s):
        """Quadratic Lagrange polynomials on {-1, 0, 1} and their slopes."""
        v = np.stack([0.5 * s * (s - 1.0), 1.0 - s * s, 0.5 * s * (s + 1.0)], axis=-1)
        d = np.stack([s - 0.5, -2.0 * s, s + 0.5], axis=-1)
        return v, d

    # cubic map (64 nodes, tensor order a + 4b + 16c at (-1 + 2a/3, ...))
    @staticmethod
    def _lag3(s):
        """Cubic Lagrange polynomials on {-1, -1/3, 1/3, 1} and their slopes."""
        nodes = (-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0)
        v, d = [], []
        for i, xi in enumerate(nodes):
            others = [xj for j, xj in enumerate(nodes) if j != i]
            den = np.prod([xi - xj for xj in others])
            v.append(np.prod([s - xj for xj in others], axis=0) / den)
            d.append(sum(np.prod([s - others[k] for k in range(3) if k != m], axis=0)
                         for m in range(3)) / den)
        return np.stack(v, axis=-1), np.stack(d, axis=-1)

    def q3_nodes(self):
        a = np.array([-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0])
        c, b, aa = np.meshgrid(a, a, a, indexing="ij")
        return np.stack([aa.ravel(), b.ravel(), c.ravel()], axis=1)

    def q3_shape(self, x):
        """(npts, 64) values of the cubic map's basis at points x."""
        v = [self._lag3(x[:, i])[0] for i in range(3)]
        return np.einsum("pa,pb,pc->pcba", v[0], v[1], v[2]).reshape(len(x), 64)

    def q3_dshape(self, x):
        vd = [self._lag3(x[:, i]) for i in range(3)]
        out = []
        for j in range(3):
            f = [vd[i][1] if i == j else vd[i][0] for i in range(3)]
            out.append(np.einsum("pa,pb,pc->pcba", f[0], f[1], f[2]).reshape(len(x), 64))
        return np.stack(out)

    def q2_shape(self, x):
        """(npts, 27) values of the quadratic map's basis at points x."""
        v = [self._lag2(x[:, i])[0] for i in range(3)]
        return np.einsum("pa,pb,pc->pcba", v[0], v[1], v[2]).reshape(len(x), 27)

    def q2_dshape(self, x):
        """(3, npts, 27): derivative along x~_j of each quadratic basis function."""
        vd = [self._lag2(x[:, i]) for i in range(3)]
        out = []
        for j in range(3):
            f = [vd[i][1] if i == j else vd[i][0] for i in range(3)]
            out.append(np.einsum("pa,pb,pc->pcba", f[0], f[1], f[2]).reshape(len(x), 27))
        return np.stack(out)


class Prism(ElementType):
    name = "pri"
    nverts = 6
    faces = [
        Face("tri", (0, 1, 2), (0, 0, -1), (1, 0, 0), (0, 1, 0), (0, 0, -1)),
        Face("tri", (3, 4, 5), (0, 0, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1)),
        Face("quad", (0, 1, 4, 3), (0, -1, 0), (1, 0, 0), (0, 0, 1), (0, -1, 0)),
        Face("quad", (1, 2, 5, 4), (0, 0, 0), (-1, 1, 0), (0, 0, 1),
             (1 / SQ2, 1 / SQ2, 0)),
        Face("quad", (0, 2, 5, 3), (-1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0)),
    ]

    def solution_points(self):
        t = tri_solution_points(self.p)
        z = gl_points(self.p)
        return np.concatenate([np.column_stack([t, np.full(len(t), zz)])
                               for zz in z])

    def basis(self, x):
        return bases.pri_basis(self.p, x)

    def grad(self, x):
        return bases.pri_grad(self.p, x)

    def volume_rule(self, n):
        return pri_rule(n)

    @staticmethod
    def _bary(x):
        return np.stack([-(x[:, 0] + x[:, 1]) / 2, (1 + x[:, 0]) / 2,
                         (1 + x[:, 1]) / 2], axis=1)

    def shape(self, x):
        lam = self._bary(x)
        zl, zh = (1 - x[:, 2:3]) / 2, (1 + x[:, 2:3]) / 2
        return np.concatenate([lam * zl, lam * zh], axis=1)

    # quadratic map (18 nodes): quadratic triangle (vertices 0, 1, 2, then the
    # midpoints of edges 01, 12, 02) times the quadratic line (z = -1, 0, 1),
    # node = triangle node + 6 * layer; the corners are nodes 0, 1, 2, 12, 13, 14
    def q2_nodes(self):
        tri = np.array([[-1, -1], [1, -1], [-1, 1], [0, -1], [0, 0], [-1, 0]], float)
        return np.concatenate([np.column_stack([tri, np.full(6, z)])
                               for z in (-1.0, 0.0, 1.0)])

    @staticmethod
    def _tri2(lam, dlam):
        """Quadratic triangle basis and its gradients from barycentrics."""
        l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
        v = np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                      4 * l0 * l1, 4 * l1 * l2, 4 * l0 * l2], axis=1)
        g = []
        for j in range(2):
            d0, d1, d2 = dlam[0][j], dlam[1][j], dlam[2][j]
            g.append(np.stack([(4 * l0 - 1) * d0, (4 * l1 - 1) * d1, (4 * l2 - 1) * d2,
                               4 * (d0 * l1 + l0 * d1), 4 * (d1 * l2 + l1 * d2),
                               4 * (d0 * l2 + l0 * d2)], axis=1))
        return v, g

    def _q2_parts(self, x):
        lam = self._bary(x)
        dlam = [(-0.5, -0.5), (0.5, 0.0), (0.0, 0.5)]
        tv, tg = self._tri2(lam, dlam)
        t = x[:, 2]
        lv = np.stack([0.5 * t * (t - 1), 1 - t * t, 0.5 * t * (t + 1)], axis=1)
        ld = np.stack([t - 0.5, -2 * t, t + 0.5], axis=1)
        return tv, tg, lv, ld

    def q2_shape(self, x):
        tv, _, lv, _ = self._q2_parts(x)
        return np.einsum("pl,pa->pla", lv, tv).reshape(len(x), 18)

    def q2_dshape(self, x):
        tv, tg, lv, ld = self._q2_parts(x)
        return np.stack([np.einsum("pl,pa->pla", lv, tg[0]).reshape(len(x), 18),
                         np.einsum("pl,pa->pla", lv, tg[1]).reshape(len(x), 18),
                         np.einsum("pl,pa->pla", ld, tv).reshape(len(x), 18)])

    # cubic map (40 nodes): the cubic triangle of _cubic_simplex (vertices
    # 0, 1, 2; edges 01, 12, 02; the centroid) times the cubic line
    # (z = -1, -1/3, 1/3, 1), node = triangle node + 10 * layer; the corners
    # are nodes 0, 1, 2, 30, 31, 32
    TRI = ((-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0))
    TRI_EDGES = ((0, 1), (1, 2), (0, 2))

    def q3_nodes(self):
        tri = _cubic_simplex_nodes(self.TRI, self.TRI_EDGES, [(0, 1, 2)])
        return np.concatenate([np.column_stack([tri, np.full(10, z)])
                               for z in (-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0)])

    def _q3_parts(self, x):
        lam = self._bary(x)
        dlam = [(-0.5, -0.5), (0.5, 0.0), (0.0, 0.5)]
        tv, tg = _cubic_simplex(lam, dlam, self.TRI_EDGES, [(0, 1, 2)])
        lv, ld = Hex._lag3(x[:, 2])
        return tv, tg, lv, ld

    def q3_shape(self, x):
        tv, _, lv, _ = self._q3_parts(x)
        return np.einsum("pl,pa->pla", lv, tv).reshape(len(x), 40)

    def q3_dshape(self, x):
        tv, tg, lv, ld = self._q3_parts(x)
        return np.stack([np.einsum("pl,pa->pla", lv, tg[0]).reshape(len(x), 40),
                         np.einsum("pl,pa->pla", lv, tg[1]).reshape(len(x), 40),
                         np.einsum("pl,pa->pla", ld, tv).reshape(len(x), 40)])

    def curl_nodes(self):
        """Nodes of the curl-form metric interpolant: the tetrahedron's face
        node set on the triangle times Gauss-Lobatto points along z (nodes
        on every face, shared with hexahedron and tetrahedron faces)."""
        t = tri_face_points(self.p)
        z = gauss_lobatto(self.p + 1)[0]
        return np.concatenate([np.column_stack([t, np.full(len(t), zz)]) for zz in z])

    def dshape(self, x):
        lam = self._bary(x)
        zl, zh = (1 - x[:, 2:3]) / 2, (1 + x[:, 2:3]) / 2
        dl = [np.tile([[-0.5, 0.5, 0.0]], (len(x), 1)),
              np.tile([[-0.5, 0.0, 0.5]], (len(x), 1))]
        d0 = np.concatenate([dl[0] * zl, dl[0] * zh], axis=1)
        d1 = np.concatenate([dl[1] * zl, dl[1] * zh], axis=1)
        d2 = np.concatenate([-0.5 * lam, 0.5 * lam], axis=1)
        return np.stack([d0, d1, d2])


class Tet(ElementType):
    name = "tet"
    nverts = 4
    faces = [
        Face("tri", (0, 1, 2), (0, 0, -1), (1, 0, 0), (0, 1, 0), (0, 0, -1)),
        Face("tri", (0, 1, 3), (0, -1, 0), (1, 0, 0), (0, 0, 1), (0, -1, 0)),
        Face("tri", (0, 2, 3), (-1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0)),
        Face("tri", (1, 2, 3), (-1, 0, 0), (-1, 1, 0), (-1, 0, 1),
             (1 / SQ3, 1 / SQ3, 1 / SQ3)),
    ]

    def solution_points(self):
        if self.p == 0:
            return np.array([[-0.5, -0.5, -0.5]])
        return tet_nodes(self.p)

    def basis(self, x):
        return bases.tet_basis(self.p, x)

    def grad(self, x):
        return bases.tet_grad(self.p, x)

    def volume_rule(self, n):
        return tet_rule(n)

    def shape(self, x):
        return np.stack([-(1 + x[:, 0] + x[:, 1] + x[:, 2]) / 2,
                         (1 + x[:, 0]) / 2, (1 + x[:, 1]) / 2,
                         (1 + x[:, 2]) / 2], axis=1)

    def dshape(self, x):
        n = len(x)
        base = np.array([[-0.5, 0.5, 0.0, 0.0], [-0.5, 0.0, 0.5, 0.0],
                         [-0.5, 0.0, 0.0, 0.5]])
        return np.stack([np.tile(base[j], (n, 1)) for j in range(3)])

    # quadratic map (10 nodes): the vertices, then the midpoints of edges
    # 01, 12, 02, 03, 13, 23
    EDGES = ((0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3))

    def q2_nodes(self):
        v = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
        return np.concatenate([v, [(v[a] + v[b]) / 2 for a, b in self.EDGES]])

    def q2_shape(self, x):
        lam = self.shape(x)                                  # barycentrics
        return np.concatenate([lam * (2 * lam - 1),
                               np.stack([4 * lam[:, a] * lam[:, b]
                                         for a, b in self.EDGES], axis=1)], axis=1)

    def q2_dshape(self, x):
        lam = self.shape(x)
        dl = self.dshape(x)                                  # (3, npts, 4)
        out = []
        for j in range(3):
            d = dl[j]
            out.append(np.concatenate(
                [(4 * lam - 1) * d,
                 np.stack([4 * (d[:, a] * lam[:, b] + lam[:, a] * d[:, b])
                           for a, b in self.EDGES], axis=1)], axis=1))
        return np.stack(out)

    # cubic map (20 nodes): _cubic_simplex on the vertices, the edges above
    # (two nodes each) and the faces 012, 013, 023, 123 (their centroids)
    FACES3 = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
    VERTS = ((-1.0, -1.0, -1.0), (1.0, -1.0, -1.0), (-1.0, 1.0, -1.0), (-1.0, -1.0, 1.0))

    def q3_nodes(self):
        return _cubic_simplex_nodes(self.VERTS, self.EDGES, self.FACES3)

    def _q3(self, x):
        dlam = [(-0.5, -0.5, -0.5), (0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]
        return _cubic_simplex(self.shape(x), dlam, self.EDGES, self.FACES3)

    def q3_shape(self, x):
        return self._q3(x)[0]

    def q3_dshape(self, x):
        return self._q3(x)[1]

    def curl_nodes(self):
        """Nodes of the curl-form metric interpolant: the warp-and-blend
        nodes (vertices, edges and faces included)."""
        return tet_nodes(self.p) if self.p > 0 else self.upts


ETYPES = {"hex": Hex, "pri": Prism, "tet": Tet}

_cache = {}


def element(name, p, family="gl"):
    """Reference element of type name and order p.  family "gll" (hexahedra
    only): Gauss-Lobatto solution points, flux points on the faces among
    them; "gl" (default): Gauss-Legendre."""
    if family not in ("gl", "gll") or (family == "gll" and name != "hex"):
        raise ValueError(f"point family {family!r} is not available for {name}")
    key = (name, p, family)
    if key not in _cache:
        _cache[key] = ETYPES[name](p, family)
    return _cache[key]
