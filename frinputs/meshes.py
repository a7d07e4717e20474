"""Seeded box meshes of linear hexahedra, prisms and tetrahedra.

Vertex order conventions (the library's documented input format):

* hex8: (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1)
  in the cell's local (i,j,k) corners;
* pri6: triangle (v0,v1,v2) at the bottom, (v3,v4,v5) above it;
* tet4: any order with positive orientation.

Boundary nodes of periodic directions are distinct nodes; periodic faces are
paired by the translation vectors returned in ``periodic``.

Curved (quadratic) elements carry, besides their corner ids, the ids of
their map nodes (``maps``): hexahedra 27 nodes in tensor order (node
a + 3 b + 9 c at reference point (-1 + a, -1 + b, -1 + c)); prisms 18 nodes,
node = triangle node + 6 * layer with triangle nodes v0, v1, v2 and the
midpoints of edges 01, 12, 02 and layers z = -1, 0, 1; tetrahedra 10 nodes,
the vertices and then the midpoints of edges 01, 12, 02, 03, 13, 23.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class MeshSpec:
    nodes: np.ndarray
    elements: dict
    periodic: list = field(default_factory=list)
    bfaces: list = field(default_factory=list)    # [(node ids, tag)]
    maps: dict = field(default_factory=dict)      # {etype: (order, map node ids)}

    def as_dict(self):
        return {"nodes": self.nodes, "elements": self.elements,
                "periodic": self.periodic, "bfaces": self.bfaces,
                "maps": self.maps}

    @property
    def n_elements(self):
        return sum(len(c) for c in self.elements.values())


def _grid_nodes(n, lo, hi):
    xs = [np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _nid(n):
    nx, ny, nz = n

    def f(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)
    return f


def _perturb(nodes, n, lo, hi, frac, seed):
    """Move nodes strictly inside the box by U(-a, a) per component,
    a = frac * h / sqrt(3), so that |displacement| <= frac * h."""
    if frac <= 0:
        return nodes
    rng = np.random.Generator(np.random.PCG64(seed))
    h = (np.asarray(hi, float) - np.asarray(lo, float)) / np.asarray(n)
    d = rng.uniform(-1.0, 1.0, size=nodes.shape) * (frac * h / np.sqrt(3.0))
    eps = 1e-12 * np.max(np.asarray(hi) - np.asarray(lo))
    inside = np.all((nodes > np.asarray(lo) + eps)
                    & (nodes < np.asarray(hi) - eps), axis=1)
    out = nodes.copy()
    out[inside] += d[inside]
    return out


def _hex_cells(n):
    nx, ny, nz = n
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                          indexing="ij")
    # element order: i fastest
    I, J, K = (a.transpose(2, 1, 0).ravel() for a in (I, J, K))
    return I, J, K


def _boundary_faces(n, f, periodic_dirs, tags):
    """Quad faces on non-periodic box sides: tags[(dir, side)]."""
    out = []
    nx, ny, nz = n
    rng = {0: (ny, nz), 1: (nx, nz), 2: (nx, ny)}
    for d in range(3):
        if d in periodic_dirs:
            continue
        for side in (0, 1):
            tag = tags[(d, side)]
            fixed = 0 if side == 0 else n[d]
            a_n, b_n = rng[d]
            for b in range(b_n):
                for a in range(a_n):
                    if d == 0:
                        ids = (f(fixed, a, b), f(fixed, a + 1, b),
                               f(fixed, a + 1, b + 1), f(fixed, a, b + 1))
                    elif d == 1:
                        ids = (f(a, fixed, b), f(a + 1, fixed, b),
                               f(a + 1, fixed, b + 1), f(a, fixed, b + 1))
                    else:
                        ids = (f(a, b, fixed), f(a + 1, b, fixed),
                               f(a + 1, b + 1, fixed), f(a, b + 1, fixed))
                    out.append((ids, tag))
    return out


def box_hex(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic=(0, 1, 2),
            perturb=0.0, seed=20240829, tags=None):
    """Box of n[0] x n[1] x n[2] hexahedra.

    periodic: directions with periodic faces; the others get boundary faces
    tagged by ``tags[(dir, side)]`` (default tag = 2*dir + side).
    perturb: fraction of the cell size by which interior nodes move.
    """
    n = tuple(int(v) for v in n)
    nodes = _perturb(_grid_nodes(n, lo, hi), n, lo, hi, perturb, seed)
    f = _nid(n)
    I, J, K = _hex_cells(n)
    conn = np.stack([f(I, J, K), f(I + 1, J, K), f(I + 1, J + 1, K),
                     f(I, J + 1, K), f(I, J, K + 1), f(I + 1, J, K + 1),
                     f(I + 1, J + 1, K + 1), f(I, J + 1, K + 1)], axis=1)
    pv = []
    for d in periodic:
        T = np.zeros(3)
        T[d] = hi[d] - lo[d]
        pv.append(T)
    if tags is None:
        tags = {(d, s): 2 * d + s for d in range(3) for s in (0, 1)}
    bf = _boundary_faces(n, f, set(periodic), tags)
    return MeshSpec(nodes, {"hex": conn.astype(np.int64)}, pv, bf)


def _orient(nodes, conn, kind):
    """Swap two vertices of every negatively oriented prism/tet."""
    x = nodes[conn]
    if kind == "tet":
        a = x[:, 1] - x[:, 0]
        b = x[:, 2] - x[:, 0]
        c = x[:, 3] - x[:, 0]
        det = np.einsum("ij,ij->i", a, np.cross(b, c))
        bad = det < 0
        conn[bad, 1], conn[bad, 2] = conn[bad, 2].copy(), conn[bad, 1].copy()
    else:
        a = x[:, 1] - x[:, 0]
        b = x[:, 2] - x[:, 0]
        c = x[:, 3] - x[:, 0]
        det = np.einsum("ij,ij->i", np.cross(a, b), c)
        bad = det < 0
        for lo_, hi_ in ((1, 2), (4, 5)):
            conn[bad, lo_], conn[bad, hi_] = (conn[bad, hi_].copy(),
                                              conn[bad, lo_].copy())
    return conn


# Kuhn (Freudenthal) split of the unit cube into six tetrahedra that share
# the main diagonal; corner index = i + 2 j + 4 k.
_KUHN = []
for _perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
    _c = [0]
    _acc = 0
    for _ax in _perm:
        _acc += (1, 2, 4)[_ax]
        _c.append(_acc)
    _KUHN.append(tuple(_c))


def mixed_box(n=40, x_pri=0.5, x_tet=0.8, perturb=0.05, seed=20240829,
              periodic_x=False):
    """Unit box of n^3 cells: hexes for x < x_pri, two prisms (split along
    the cell's xy diagonal, axis along z) for x_pri <= x < x_tet and six
    Kuhn tetrahedra for x >= x_tet.  y and z are periodic.  Quad faces and
    triangular tet faces cannot conform, so both sides of the plane
    x = x_tet (when tets meet hexes or prisms there) are boundary faces:
    tag 2 on the quad side, tag 3 on the tet side.  x = 0 and x = 1 are
    boundary faces with tags 0 and 1, or periodic when ``periodic_x`` (valid
    only when the faces at x = 0 and x = 1 are of the same kind)."""
    N = (n, n, n)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    nodes = _grid_nodes(N, lo, hi)
    f = _nid(N)
    i_pri = int(round(x_pri * n))
    i_tet = int(round(x_tet * n))
    nodes = _perturb(nodes, N, lo, hi, perturb, seed)
    I, J, K = _hex_cells(N)
    corner = [f(I + (c & 1), J + ((c >> 1) & 1), K + ((c >> 2) & 1))
              for c in range(8)]
    c = np.stack(corner, axis=1)
    hexes = c[I < i_pri][:, [0, 1, 3, 2, 4, 5, 7, 6]]
    cp = c[(I >= i_pri) & (I < i_tet)]
    pris = np.empty((2 * len(cp), 6), np.int64)
    pris[0::2] = cp[:, [0, 1, 3, 4, 5, 7]]
    pris[1::2] = cp[:, [0, 3, 2, 4, 7, 6]]
    ct = c[I >= i_tet]
    tets = np.empty((6 * len(ct), 4), np.int64)
    for q, kt in enumerate(_KUHN):
        tets[q::6] = ct[:, list(kt)]
    pris = _orient(nodes, pris, "pri")
    tets = _orient(nodes, tets, "tet")
    elements = {"hex": hexes, "pri": pris, "tet": tets}
    plane = {k: np.nonzero(np.abs(_grid_nodes(N, lo, hi)[:, 0] - k / n)
                           < 1e-12)[0] for k in (0, n, i_tet)}
    bf = []
    pv = [np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])]
    if periodic_x:
        pv.append(np.array([1.0, 0.0, 0.0]))
    else:
        bf += _plane_faces(elements, plane[0], None, 0)
        bf += _plane_faces(elements, plane[n], None, 1)
    if 0 < i_tet < n and (i_pri > 0 or i_tet > i_pri):
        bf += _plane_faces({"hex": hexes, "pri": pris}, plane[i_tet], None, 2)
        bf += _plane_faces({"tet": tets}, plane[i_tet], None, 3)
    return MeshSpec(nodes, elements, pv, bf)


def _plane_faces(elements, plane_nodes, _unused, tag):
    """Element faces whose vertices all lie in a plane given by its node
    ids: 4 such vertices of a hex or prism, 3 of a tet."""
    on = set(int(v) for v in plane_nodes)
    out = []
    for kind, conn in elements.items():
        want = 3 if kind == "tet" else 4
        for ev in conn:
            vs = [int(v) for v in ev if int(v) in on]
            if len(vs) == want:
                out.append((tuple(vs), tag))
    return out


def curved_box_hex(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic=(0, 1, 2),
                   amp=0.05, tags=None, order=2):
    """Box of n[0] x n[1] x n[2] curved hexahedra with quadratic (order 2,
    27 nodes) or cubic (order 3, 64 nodes: node a + 4b + 16c at reference
    point (-1 + 2a/3, -1 + 2b/3, -1 + 2c/3)) maps.

    The (order n + 1)^3 lattice of map nodes is displaced by d_k = amp h_k
    (sin(pi n_{k+1} X_{k+1}) + sin(pi n_{k+2} X_{k+2})) (1 + cos(2 pi n_k
    X_k) / 2) (X the box coordinates scaled to [0, 1], indices cyclic).
    Corners stay on the grid (the sines vanish there), the field is the same
    on opposite box sides (faces pair by their corner ids or periodic
    translation), and each component depends on all three coordinates, so
    the map's cofactors are of high degree.
    """
    n = tuple(int(v) for v in n)
    o = int(order)
    m = tuple(o * v for v in n)
    lo_a, hi_a = np.asarray(lo, float), np.asarray(hi, float)
    nodes = _grid_nodes(m, lo, hi)
    L = hi_a - lo_a
    h = L / np.asarray(n, float)
    X = (nodes - lo_a) / L
    sn = [np.sin(np.pi * n[k] * X[:, k]) for k in range(3)]
    d = np.stack([h[k] * (sn[(k + 1) % 3] + sn[(k + 2) % 3])
                  * (1.0 + 0.5 * np.cos(2.0 * np.pi * n[k] * X[:, k]))
                  for k in range(3)], axis=1)
    nodes = nodes + amp * d
    g = _nid(m)
    I, J, K = _hex_cells(n)
    a = np.arange(o + 1)
    A, B, C = np.meshgrid(a, a, a, indexing="ij")
    A, B, C = (v.transpose(2, 1, 0).ravel() for v in (A, B, C))   # a fastest
    hmap = g(o * I[:, None] + A[None, :], o * J[:, None] + B[None, :],
             o * K[:, None] + C[None, :])
    q = o + 1
    corner = hmap[:, [0, o, o + q * o, q * o, q * q * o, o + q * q * o,
                      o + q * o + q * q * o, q * o + q * q * o]]
    pv = []
    for dd in periodic:
        T = np.zeros(3)
        T[dd] = hi[dd] - lo[dd]
        pv.append(T)
    if tags is None:
        tags = {(dd, s_): 2 * dd + s_ for dd in range(3) for s_ in (0, 1)}
    # boundary faces on the map lattice: corner ids of each quad
    fo = lambda i, j, k: g(o * i, o * j, o * k)  # noqa: E731
    bf = _boundary_faces(n, fo, set(periodic), tags)
    return MeshSpec(nodes, {"hex": corner.astype(np.int64)}, pv, bf,
                    {"hex": (o, hmap.astype(np.int64))})


# reference coordinates of the quadratic map nodes of each element type, in
# the library's node order (see the module docstring)
_Q2_REF = {
    "hex": np.array([[-1 + a, -1 + b, -1 + c] for c in range(3) for b in range(3)
                     for a in range(3)], float),
    "pri": np.array([[x, y, z] for z in (-1.0, 0.0, 1.0)
                     for x, y in ((-1, -1), (1, -1), (-1, 1), (0, -1), (0, 0), (-1, 0))],
                    float),
    "tet": np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1],
                     [0, -1, -1], [0, 0, -1], [-1, 0, -1], [-1, -1, 0],
                     [0, -1, 0], [-1, 0, 0]], float),
}


def _simplex_cubic_ref(verts, edges, faces):
    v = np.asarray(verts, float)
    out = list(v)
    for a, b in edges:
        out += [(2 * v[a] + v[b]) / 3, (v[a] + 2 * v[b]) / 3]
    out += [v[list(f)].mean(axis=0) for f in faces]
    return np.array(out)


# reference coordinates of the cubic map nodes, in the library's node order:
# hexahedra a + 4b + 16c at (-1 + 2a/3, ...); prisms triangle node + 10 *
# layer (triangle: vertices, two nodes on each of the edges 01, 12, 02 -- the
# one nearer the edge's first vertex first -- and the centroid; layers z =
# -1, -1/3, 1/3, 1); tetrahedra: vertices, two nodes on each of the edges
# 01, 12, 02, 03, 13, 23, the centroids of the faces 012, 013, 023, 123
_THIRDS = (-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0)
_TRI3 = _simplex_cubic_ref([(-1, -1), (1, -1), (-1, 1)], [(0, 1), (1, 2), (0, 2)],
                           [(0, 1, 2)])
_Q3_REF = {
    "hex": np.array([[a, b, c] for c in _THIRDS for b in _THIRDS for a in _THIRDS]),
    "pri": np.array([[x, y, z] for z in _THIRDS for x, y in _TRI3]),
    "tet": _simplex_cubic_ref([(-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)],
                              [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)],
                              [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]),
}


def _linear_shape(kind, x):
    """Linear (vertex) shape functions of the reference element at x (n, 3)."""
    if kind == "hex":
        s = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                      [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float)
        return np.prod(1 + x[:, None, :] * s[None], axis=2) / 8.0
    if kind == "pri":
        lam = np.stack([-(x[:, 0] + x[:, 1]) / 2, (1 + x[:, 0]) / 2, (1 + x[:, 1]) / 2], 1)
        zl, zh = (1 - x[:, 2:3]) / 2, (1 + x[:, 2:3]) / 2
        return np.concatenate([lam * zl, lam * zh], axis=1)
    return np.stack([-(1 + x[:, 0] + x[:, 1] + x[:, 2]) / 2, (1 + x[:, 0]) / 2,
                     (1 + x[:, 1]) / 2, (1 + x[:, 2]) / 2], axis=1)


def curved_mixed_box(n=8, x_pri=0.34, x_tet=0.67, amp=0.05, periodic_x=False,
                     order=2):
    """The mixed_box layout (hexahedra, prisms, Kuhn tetrahedra; no vertex
    jitter) with curved maps on every element: order 2, 27-node hexahedra,
    18-node prisms, 10-node tetrahedra; order 3, 64-node hexahedra, 40-node
    prisms, 20-node tetrahedra.  All map nodes lie on the (order n + 1)^3
    lattice of the cells' 1/order points (vertices, edge, face and cell
    points), displaced by the smooth field of curved_box_hex (corners stay on
    the grid), so neighbouring elements share their face nodes."""
    o = int(order)
    coarse = mixed_box(n=n, x_pri=x_pri, x_tet=x_tet, perturb=0.0,
                       periodic_x=periodic_x)
    m = (o * n, o * n, o * n)
    lat = _grid_nodes(m, (0, 0, 0), (1, 1, 1))
    h = np.full(3, 1.0 / n)
    X = lat
    sn = [np.sin(np.pi * n * X[:, k]) for k in range(3)]
    d = np.stack([h[k] * (sn[(k + 1) % 3] + sn[(k + 2) % 3])
                  * (1.0 + 0.5 * np.cos(2.0 * np.pi * n * X[:, k]))
                  for k in range(3)], axis=1)
    nodes = lat + amp * d
    g = _nid(m)
    # lattice coordinates of the coarse grid's nodes
    ci = np.arange((n + 1) ** 3)
    cl = o * np.stack([ci % (n + 1), (ci // (n + 1)) % (n + 1),
                       ci // (n + 1) ** 2], axis=1)

    def lid(c):
        return g(c[..., 0], c[..., 1], c[..., 2])
    elements, maps = {}, {}
    for kind, conn in coarse.elements.items():
        if len(conn) == 0:
            continue
        Nl = _linear_shape(kind, (_Q2_REF if o == 2 else _Q3_REF)[kind])  # (n_map, n_vert)
        vc = cl[conn]                                      # (ne, n_vert, 3)
        q = np.einsum("mv,evk->emk", Nl, vc)
        qi = np.rint(q).astype(np.int64)
        assert np.abs(q - qi).max() < 1e-9
        maps[kind] = (o, lid(qi))
        elements[kind] = lid(vc)
    bf = [(tuple(int(lid(cl[v])) for v in ids), tag) for ids, tag in coarse.bfaces]
    return MeshSpec(nodes, elements, coarse.periodic, bf, maps)
