"""Mesh geometry and interface pairing for the oracle (test infrastructure only).

Section 2: the domain is tessellated into conforming elements, each mapped
from its reference element by x = M_n(x~) with Jacobian J = dM/dx~ and
transformed flux f~ = J J^{-1} f.  Flux points of adjoining elements conform
at interfaces (Section 2), so every flux point of an interior face has one
partner with the same physical coordinates.

* metrics: S = det(J) J^{-1} at solution and flux points, straight from the
  vertex map (linear elements, Section 3.4: metrics from the vertices);
* curved elements (quadratic maps: 27-node hexahedra, 18-node prisms,
  10-node tetrahedra, "Curved Elements" of Section 3.4): the conservative
  metric, i.e. the curl form S[i][n] = -(curl_xi I(X_l grad_xi X_m))_i,
  (n, m, l) cyclic, with I the order-p interpolation on a node set with
  nodes on every face, evaluated at the solution and flux points; det J is
  the map's own;
* surface normal at a flux point: S^T n~ (Nanson), split into its magnitude
  and the physical unit normal;
* faces are paired by their vertex sets; faces left over are paired
  periodically when a translation vector maps one face centroid onto the
  other; the rest must be listed as boundary faces (else the mesh is
  rejected as non-conforming);
* flux points of a paired face are matched by physical coordinates.
"""
import numpy as np
from scipy.spatial import cKDTree

from .elements import element
from .polys import dlagrange_matrix, gauss_lobatto, lagrange_matrix

ETYPE_ORDER = ("hex", "pri", "tet")


class MeshError(ValueError):
    pass


def _map_fns(el, order):
    """Shape functions (values, derivatives) of an element map of `order`."""
    if order == 3:
        return el.q3_shape, el.q3_dshape
    return el.q2_shape, el.q2_dshape


def curl_metric(el, Xm, pts, order=2):
    """Conservative (curl-form) metric of quadratic maps at the reference
    points pts.  Xm: (ne, n_map, 3) map nodes.  The fields
    w^n_j = X_l dX_m/dxi_j ((n, m, l) cyclic) are interpolated by the
    order-p polynomial of the element's solution space on a node set with
    nodes on every face (a face's normal component depends on that face
    only, so neighbours agree): the (p+1)^3 Gauss-Lobatto nodes on
    hexahedra, el.curl_nodes() on prisms and tetrahedra; then
    S[i][n] = -(curl_xi of it)_i at pts.  Returns S[e, q, i, n]
    (= det J dxi_i/dx_n).  order: 2 (quadratic maps) or 3 (cubic maps:
    64-node hexahedra, 40-node prisms, 20-node tetrahedra)."""
    shape, dshape = _map_fns(el, order)
    if el.name != "hex":
        G = el.curl_nodes()
        Vi = np.linalg.inv(el.basis(G))
        dB = [gj @ Vi for gj in el.grad(pts)]                    # (npts, nG)
        X = np.einsum("pv,evk->epk", shape(G), Xm)
        dX = np.einsum("jpv,evk->epjk", dshape(G), Xm)
        S = np.zeros((Xm.shape[0], len(pts), 3, 3))
        for n in range(3):
            m, l = (n + 1) % 3, (n + 2) % 3
            w = X[:, :, l, None] * dX[:, :, :, m]
            for i in range(3):
                j, k = (i + 1) % 3, (i + 2) % 3
                S[:, :, i, n] = -(np.einsum("pg,eg->ep", dB[j], w[:, :, k])
                                  - np.einsum("pg,eg->ep", dB[k], w[:, :, j]))
        return S
    g, _ = gauss_lobatto(el.p + 1)
    n1 = len(g)
    c, b, a = np.meshgrid(g, g, g, indexing="ij")
    G = np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)      # x~_0 fastest
    X = np.einsum("pv,evk->epk", shape(G), Xm)
    dX = np.einsum("jpv,evk->epjk", dshape(G), Xm)              # d x_k / d xi_j
    L = [lagrange_matrix(g, pts[:, i]) for i in range(3)]
    dL = [dlagrange_matrix(g, pts[:, i]) for i in range(3)]

    def tensor(f0, f1, f2):
        return np.einsum("pa,pb,pc->pcba", f0, f1, f2).reshape(len(pts), n1 ** 3)
    dB = [tensor(*(dL[i] if i == j else L[i] for i in range(3))) for j in range(3)]
    S = np.zeros((Xm.shape[0], len(pts), 3, 3))
    for n in range(3):
        m, l = (n + 1) % 3, (n + 2) % 3
        w = X[:, :, l, None] * dX[:, :, :, m]                    # w_j = X_l dX_m/dxi_j
        for i in range(3):
            j, k = (i + 1) % 3, (i + 2) % 3
            S[:, :, i, n] = -(np.einsum("pg,eg->ep", dB[j], w[:, :, k])
                              - np.einsum("pg,eg->ep", dB[k], w[:, :, j]))
    return S


class FRMesh:
    """Geometry + connectivity of an FR discretisation of order p.

    spec: dict with keys
      nodes    (n, 3) float64
      elements {etype: (n_e, n_v) int64 connectivity}
      periodic list of translation 3-vectors (may be empty)
      bfaces   list of (node-id tuple, tag) for boundary faces
    """

    def __init__(self, spec, p, family="gl"):
        self.p = p
        self.family = family
        nodes = np.asarray(spec["nodes"], np.float64)
        self.types = [t for t in ETYPE_ORDER
                      if t in spec["elements"] and len(spec["elements"][t])]
        if family == "gll" and "pri" in self.types:
            # a hexahedron's Gauss-Lobatto quad faces cannot meet a prism's
            # Gauss-Legendre ones
            raise MeshError("the Gauss-Lobatto family needs a mesh without prisms")
        self.el = {t: element(t, p, family if t == "hex" else "gl")
                   for t in self.types}
        self.conn = {t: np.asarray(spec["elements"][t], np.int64)
                     for t in self.types}
        self.verts = {t: nodes[self.conn[t]] for t in self.types}
        self.ne = {t: len(self.conn[t]) for t in self.types}
        self.upts_x, self.S_u, self.detJ = {}, {}, {}
        self.fpts_x, self.fnorm, self.fmag = {}, {}, {}
        maps = spec.get("maps", {}) or {}
        self.curved = {}
        self._Xm = {}
        self._morder = {}
        for t in self.types:
            el, V = self.el[t], self.verts[t]
            morder, mconn = maps.get(t, (1, None))
            self.curved[t] = morder >= 2
            if morder in (2, 3):
                shape, dshape = _map_fns(el, morder)
                Xm = nodes[np.asarray(mconn, np.int64)]
                self._Xm[t] = Xm
                self._morder[t] = morder
                self.upts_x[t] = np.einsum("pv,evk->epk", shape(el.upts), Xm)
                self.S_u[t] = curl_metric(el, Xm, el.upts, morder)
                dX = np.einsum("jpv,evk->epjk", dshape(el.upts), Xm)
                self.detJ[t] = np.linalg.det(dX)
                self.fpts_x[t] = np.einsum("pv,evk->epk", shape(el.fpts), Xm)
                Sf = curl_metric(el, Xm, el.fpts, morder)
            elif morder == 1:
                self.upts_x[t] = el.map_points(V, el.upts)
                self.S_u[t], self.detJ[t] = el.metrics(V, el.upts)
                self.fpts_x[t] = el.map_points(V, el.fpts)
                Sf, _ = el.metrics(V, el.fpts)
            else:
                raise MeshError(f"map order {morder} not implemented")
            if np.any(self.detJ[t] <= 0):
                raise MeshError(f"non-positive Jacobian in {t} elements")
            nv = np.einsum("epij,pi->epj", Sf, el.fpts_norm)
            mag = np.linalg.norm(nv, axis=2)
            self.fmag[t] = mag
            self.fnorm[t] = nv / mag[:, :, None]
        # global flux-point numbering: off[t] + e * nfpts + i
        self.foff, n = {}, 0
        for t in self.types:
            self.foff[t] = n
            n += self.ne[t] * self.el[t].nfpts
        self.nfpts_total = n
        self._pair(nodes, spec.get("periodic", []), spec.get("bfaces", []))

    def metric_at(self, t, pts):
        """S = det J J^{-1} of every element of type t at reference points
        pts, in the form the mesh uses (curl form on curved elements, the
        map's cross products otherwise).  Shape (ne, npts, 3, 3)."""
        if self.curved[t]:
            return curl_metric(self.el[t], self._Xm[t], pts, self._morder[t])
        return self.el[t].metrics(self.verts[t], pts)[0]

    def gidx(self, t, e, i):
        return self.foff[t] + e * self.el[t].nfpts + i

    def flat(self, arrs):
        """Concatenate per-type (n_e, n_f, ...) arrays into global order."""
        return np.concatenate([arrs[t].reshape((-1,) + arrs[t].shape[2:])
                               for t in self.types])

    def _pair(self, nodes, periodic, bfaces):
        recs = []           # (t, e, f, key tuple)
        keys = []
        for t in self.types:
            el = self.el[t]
            for f, face in enumerate(el.faces):
                ids = np.sort(self.conn[t][:, list(face.verts)], axis=1)
                if ids.shape[1] == 3:
                    ids = np.concatenate([np.full((len(ids), 1), -1), ids],
                                         axis=1)
                keys.append(ids)
                recs.append(np.stack([np.full(len(ids), ETYPE_ORDER.index(t)),
                                      np.arange(len(ids)),
                                      np.full(len(ids), f)], axis=1))
        keys = np.concatenate(keys)
        recs = np.concatenate(recs)
        order = np.lexsort(keys.T[::-1])
        ks = keys[order]
        same = np.all(ks[1:] == ks[:-1], axis=1)
        if np.any(same[1:] & same[:-1]):
            raise MeshError("a face is shared by more than two elements")
        matched = np.zeros(len(keys), bool)
        face_pairs = []     # (recL, recR, T)
        for i in np.nonzero(same)[0]:
            a, b = order[i], order[i + 1]
            matched[a] = matched[b] = True
            face_pairs.append((recs[a], recs[b], np.zeros(3)))
        # periodic pairing of left-over faces by centroid translation
        left = np.nonzero(~matched)[0]
        cent = np.array([nodes[[v for v in keys[i] if v >= 0]].mean(axis=0)
                         for i in left]).reshape(-1, 3)
        scale = np.ptp(nodes, axis=0).max()
        tol = 1e-8 * scale
        used = np.zeros(len(left), bool)
        if len(left) and len(periodic):
            tree = cKDTree(cent)
            for T in periodic:
                T = np.asarray(T, np.float64)
                d, j = tree.query(cent + T)
                for i in np.nonzero(d < tol)[0]:
                    if used[i] or used[j[i]]:
                        continue
                    if keys[left[i]][0] == -1 and keys[left[j[i]]][0] != -1:
                        raise MeshError("periodic tri/quad mismatch")
                    used[i] = used[j[i]] = True
                    face_pairs.append((recs[left[i]], recs[left[j[i]]], T))
        # boundary faces
        bkey = {}
        for ids, tag in bfaces:
            k = tuple(sorted(ids))
            if len(k) == 3:
                k = (-1,) + k
            bkey[k] = tag
        bnd = []
        for i in np.nonzero(~used)[0]:
            k = tuple(int(v) for v in keys[left[i]])
            if k not in bkey:
                raise MeshError("unmatched face (non-conforming mesh)")
            bnd.append((recs[left[i]], bkey[k]))
        self._pair_points(face_pairs, bnd, tol)

    def _pair_points(self, face_pairs, bnd, tol):
        # Orientation of every interface: its "-" side (pair_l) is the
        # element with the lower global index (types in the order hex, pri,
        # tet, then element number), the lower face number for an element
        # paired with itself.  Upwind-biased schemes (LDG) depend on it.
        eoff, n = {}, 0
        for t in self.types:
            eoff[t] = n
            n += self.ne[t]
        gl, gr = [], []
        for rl, rr, T in face_pairs:
            kl = (eoff[ETYPE_ORDER[rl[0]]] + rl[1], rl[2])
            kr = (eoff[ETYPE_ORDER[rr[0]]] + rr[1], rr[2])
            if kr < kl:
                rl, rr, T = rr, rl, -np.asarray(T, float)
            tl, tr = ETYPE_ORDER[rl[0]], ETYPE_ORDER[rr[0]]
            il = self.el[tl].face_fpts[rl[2]]
            ir = self.el[tr].face_fpts[rr[2]]
            if len(il) != len(ir):
                raise MeshError("face kinds differ across an interface")
            xl = self.fpts_x[tl][rl[1], il] + T
            xr = self.fpts_x[tr][rr[1], ir]
            d = np.linalg.norm(xl[:, None, :] - xr[None, :, :], axis=2)
            m = np.argmin(d, axis=1)
            if (d[np.arange(len(il)), m].max() > tol
                    or len(set(m.tolist())) != len(il)):
                raise MeshError("flux points do not conform across a face")
            gl.append(self.gidx(tl, rl[1], il))
            gr.append(self.gidx(tr, rr[1], ir[m]))
        self.pair_l = np.concatenate(gl) if gl else np.zeros(0, np.int64)
        self.pair_r = np.concatenate(gr) if gr else np.zeros(0, np.int64)
        bg, btag = [], []
        for rec, tag in bnd:
            t = ETYPE_ORDER[rec[0]]
            i = self.el[t].face_fpts[rec[2]]
            bg.append(self.gidx(t, rec[1], i))
            btag.append(np.full(len(i), tag))
        self.bnd_g = np.concatenate(bg) if bg else np.zeros(0, np.int64)
        self.bnd_tag = np.concatenate(btag) if btag else np.zeros(0, np.int64)
        fn = self.flat(self.fnorm)
        fm = self.flat(self.fmag)
        self.fn_all, self.fm_all = fn, fm
        if len(self.pair_l):
            # magnitudes may differ (they scale different reference faces);
            # the physical unit normals must be opposite
            dn = np.abs(fn[self.pair_l] + fn[self.pair_r]).max()
            if dn > 1e-8:
                raise MeshError("interface normals do not match")
