"""Pins for the oracle's curved (quadratic) elements and their conservative
metric ("Curved Elements", Section 3.4): the curl form keeps a uniform flow
uniform on curved grids, including where the pointwise cross-product metric
does not (the comparison the paper draws in its free-stream figure); it is
exact for straight elements written as quadratic maps, discretely
divergence free, and conservative across curved faces.

The pointwise metric is swapped in while the mesh is built, so that the
interface normals come from it too.  So built, it keeps free stream on
quadratic hexahedra for p >= 2 as well; it fails at p = 1 and, at p = 2, on
prisms and tetrahedra -- those are the discriminating cases."""
import numpy as np
import pytest

import oracle.mesh as omesh
from frinputs import box_hex, curved_box_hex, curved_mixed_box, ics, mixed_box
from oracle.fr import FRSystem
from oracle.mesh import FRMesh


def _uniform(m):
    el = m.el["hex"]
    u = np.zeros((m.ne["hex"], el.nupts, 5))
    v = np.array([0.5, 0.3, 0.2])
    u[..., 0] = 1.0
    u[..., 1:4] = v
    u[..., 4] = 1.0 / 0.4 + 0.5 * v @ v
    return {"hex": u}


def _pointwise_metric(el, Xm, pts, order=2):
    """S = det J J^{-1} from the cross products of the map's columns."""
    a = np.einsum("jpv,evk->epjk", el.q2_dshape(pts), Xm)
    return np.stack([np.cross(a[:, :, 1], a[:, :, 2]),
                     np.cross(a[:, :, 2], a[:, :, 0]),
                     np.cross(a[:, :, 0], a[:, :, 1])], axis=2)


def _mesh(spec, p, pointwise=False):
    if not pointwise:
        return FRMesh(spec.as_dict(), p)
    orig = omesh.curl_metric
    omesh.curl_metric = _pointwise_metric
    try:
        return FRMesh(spec.as_dict(), p)
    finally:
        omesh.curl_metric = orig


def _jittered(spec, n, frac=0.1, seed=3, order=2):
    """Generic maps: the map nodes strictly inside the box that are not cell
    corners moved by U(-a, a) per component, a = frac h / order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = order * n + 1
    ids = np.arange(len(spec.nodes))
    ijk = np.stack([ids % m, (ids // m) % m, ids // (m * m)], axis=1)
    mv = np.all((ijk > 0) & (ijk < m - 1), axis=1) & np.any(ijk % order != 0, axis=1)
    spec.nodes = spec.nodes.copy()
    spec.nodes[mv] += rng.uniform(-1, 1, (mv.sum(), 3)) * frac / (order * n)
    return spec


UNIFORM_BCS = {k: ("state", 1.0, 0.5, 0.3, 0.2, 1.0) for k in range(6)}


def _free_stream_residual(m, physics="euler"):
    u = {t: ics.uniform(m.upts_x[t].reshape(-1, 3), vel=(0.5, 0.3, 0.2)).reshape(m.ne[t], -1, 5)
         for t in m.types}
    r = FRSystem(m, physics, mu=0.01, bcs=UNIFORM_BCS).rhs(u)
    return max(np.abs(v).max() for v in r.values())


@pytest.mark.parametrize("p", [2, 3])
def test_curl_metric_is_discretely_divergence_free(p):
    m = FRMesh(curved_box_hex((3, 3, 3)).as_dict(), p)
    el, S = m.el["hex"], m.S_u["hex"]
    for n in range(3):
        div = sum(np.einsum("pq,eq->ep", el.D[i], S[:, :, i, n]) for i in range(3))
        assert np.abs(div).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_free_stream_kept_by_conservative_metric(p):
    spec = _jittered(curved_box_hex((3, 3, 3)), 3)
    assert _free_stream_residual(_mesh(spec, p)) < 1e-10     # residual scale ~1e2


def test_pointwise_metric_loses_free_stream_where_curl_form_keeps_it():
    """Quadratic hexahedra at p = 1 and curved prisms / tetrahedra at p = 2:
    the pointwise metric leaves a residual of order one, the curl form
    round-off."""
    hexes = _jittered(curved_box_hex((3, 3, 3)), 3)
    assert _free_stream_residual(_mesh(hexes, 1)) < 1e-11
    assert _free_stream_residual(_mesh(hexes, 1, pointwise=True)) > 1e-2
    mixed = _jittered(curved_mixed_box(n=3), 3)
    assert _free_stream_residual(_mesh(mixed, 2)) < 1e-10
    assert _free_stream_residual(_mesh(mixed, 2, pointwise=True)) > 1e-2


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_free_stream_on_curved_mixed_mesh(p, physics):
    """Quadratic 27-node hexahedra, 18-node prisms and 10-node tetrahedra
    with generic (jittered) maps."""
    spec = _jittered(curved_mixed_box(n=3), 3)
    assert _free_stream_residual(_mesh(spec, p), physics) < 1e-10


@pytest.mark.parametrize("p", [2, 3])
def test_curl_metric_equals_analytic_on_trilinear_elements(p):
    """A perturbed trilinear hexahedron written as a 27-node map: its
    cofactors are quadratic, so the order-p curl form reproduces the
    analytic metric exactly."""
    lin = box_hex((2, 2, 2), perturb=0.1)
    ml = FRMesh(lin.as_dict(), p)
    el = ml.el["hex"]
    V = lin.nodes[lin.elements["hex"]]                   # (ne, 8, 3)
    g = np.array([-1.0, 0.0, 1.0])
    C, B, A = np.meshgrid(g, g, g, indexing="ij")
    ref = np.stack([A.ravel(), B.ravel(), C.ravel()], axis=1)
    Xq = el.map_points(V, ref)                           # (ne, 27, 3) on the trilinear map
    nodes = np.concatenate([lin.nodes, Xq.reshape(-1, 3)])
    mids = len(lin.nodes) + np.arange(Xq.shape[0] * 27).reshape(-1, 27)
    spec = dict(lin.as_dict())
    spec["nodes"] = nodes
    spec["maps"] = {"hex": (2, mids)}
    mc = FRMesh(spec, p)
    scale = np.abs(ml.S_u["hex"]).max()
    assert np.abs(mc.S_u["hex"] - ml.S_u["hex"]).max() < 1e-13 * scale
    assert np.abs(mc.fmag["hex"] - ml.fmag["hex"]).max() < 1e-13 * scale


def test_conservation_on_curved_periodic_mesh():
    """sum_e sum_q w_q J_q R_q = 0: the interface fluxes of both sides of a
    curved face cancel (watertight normals)."""
    m = FRMesh(curved_box_hex((3, 3, 3)).as_dict(), 3)
    sysm = FRSystem(m, "ns", mu=0.02)
    el = m.el["hex"]
    x = m.upts_x["hex"]
    u = {"hex": ics.taylor_green(2 * np.pi * x.reshape(-1, 3), mach=0.3).reshape(x.shape[0], -1, 5)}
    R = sysm.rhs(u)["hex"]
    tot = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], R)
    scale = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], np.abs(R))
    assert np.all(np.abs(tot) < 1e-13 * scale.max()), tot / scale.max()


@pytest.mark.parametrize("kind", ["pri", "tet"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_curl_metric_equals_analytic_on_straight_simplices(kind, p):
    """Straight prisms and tetrahedra written as quadratic maps: the curl form
    equals the map's analytic metric at solution and flux points."""
    lin = mixed_box(n=2, x_pri=0.0 if kind == "pri" else 1.0, x_tet=1.0 if kind == "pri" else 0.0,
                    perturb=0.05)
    ml = FRMesh(lin.as_dict(), p)
    el = ml.el[kind]
    V = lin.nodes[lin.elements[kind]]
    Xq = el.map_points(V, el.q2_nodes())
    nmap = Xq.shape[1]
    nodes = np.concatenate([lin.nodes, Xq.reshape(-1, 3)])
    mids = len(lin.nodes) + np.arange(Xq.shape[0] * nmap).reshape(-1, nmap)
    spec = dict(lin.as_dict())
    spec["nodes"] = nodes
    spec["maps"] = {kind: (2, mids)}
    mc = FRMesh(spec, p)
    scale = np.abs(ml.S_u[kind]).max()
    assert np.abs(mc.S_u[kind] - ml.S_u[kind]).max() < 1e-13 * scale
    assert np.abs(mc.fmag[kind] - ml.fmag[kind]).max() < 1e-13 * scale
    assert np.abs(mc.detJ[kind] - ml.detJ[kind]).max() < 1e-13 * np.abs(ml.detJ[kind]).max()


@pytest.mark.parametrize("p", [2, 3])
def test_curl_metric_of_simplices_is_discretely_divergence_free(p):
    m = FRMesh(_jittered(curved_mixed_box(n=3), 3).as_dict(), p)
    for t in ("pri", "tet"):
        el, S = m.el[t], m.S_u[t]
        for n in range(3):
            div = sum(np.einsum("pq,eq->ep", el.D[i], S[:, :, i, n]) for i in range(3))
            assert np.abs(div).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("layout", [(0.0, 1.0), (0.0, 0.0), (0.5, 1.0)])
def test_conservation_on_curved_periodic_mixed_meshes(layout):
    """All prisms, all tetrahedra, hexahedra | prisms; curved and periodic."""
    spec = _jittered(curved_mixed_box(n=3, x_pri=layout[0], x_tet=layout[1],
                                      periodic_x=True), 3)
    m = FRMesh(spec.as_dict(), 3)
    u = {t: ics.flow3d(m.upts_x[t].reshape(-1, 3)).reshape(m.ne[t], -1, 5) for t in m.types}
    R = FRSystem(m, "ns", mu=0.02).rhs(u)
    tot = sum(np.einsum("q,eq,eqk->k", m.el[t].W, m.detJ[t], R[t]) for t in m.types)
    scale = sum(np.einsum("q,eq,eqk->k", m.el[t].W, m.detJ[t], np.abs(R[t])) for t in m.types)
    assert np.all(np.abs(tot) < 1e-13 * scale.max()), tot / scale.max()


# ---------------------------------------------------------------- cubic maps
def _pointwise3(el, Xm, pts, order=3):
    a = np.einsum("jpv,evk->epjk", el.q3_dshape(pts), Xm)
    return np.stack([np.cross(a[:, :, 1], a[:, :, 2]),
                     np.cross(a[:, :, 2], a[:, :, 0]),
                     np.cross(a[:, :, 0], a[:, :, 1])], axis=2)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cubic_hexahedra_free_stream_and_conservation(p):
    spec = _jittered(curved_box_hex((3, 3, 3), order=3), 3, order=3)
    m = FRMesh(spec.as_dict(), p)
    assert _free_stream_residual(m) < 1e-10
    u = {"hex": ics.flow3d(m.upts_x["hex"].reshape(-1, 3)).reshape(m.ne["hex"], -1, 5)}
    R = FRSystem(m, "ns", mu=0.02).rhs(u)["hex"]
    el = m.el["hex"]
    tot = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], R)
    scale = np.einsum("q,eq,eqk->k", el.W, m.detJ["hex"], np.abs(R))
    assert np.all(np.abs(tot) < 1e-13 * scale.max())


@pytest.mark.parametrize("p", [2, 3])
def test_cubic_pointwise_metric_loses_free_stream(p):
    """Generic (jittered) cubic maps: the pointwise metric loses free stream
    by O(1) at p = 2 and 3, the curl form keeps it."""
    spec = _jittered(curved_box_hex((3, 3, 3), order=3), 3, order=3)
    orig = omesh.curl_metric
    omesh.curl_metric = lambda el, Xm, pts, order=2: _pointwise3(el, Xm, pts)
    try:
        mx = FRMesh(spec.as_dict(), p)
    finally:
        omesh.curl_metric = orig
    assert _free_stream_residual(mx) > 1e-2
    assert _free_stream_residual(FRMesh(spec.as_dict(), p)) < 1e-10


@pytest.mark.parametrize("p", [2, 3, 4])
def test_quadratic_map_written_as_cubic_gives_the_same_metric(p):
    """Cubic map nodes placed on a quadratic map: the same geometry, so the
    same curl-form metric, det J and points."""
    q = curved_box_hex((2, 2, 2))
    m2 = FRMesh(q.as_dict(), p)
    el = m2.el["hex"]
    X2 = q.nodes[q.maps["hex"][1]]
    X3 = np.einsum("pv,evk->epk", el.q2_shape(el.q3_nodes()), X2)   # (ne, 64, 3)
    nodes = np.concatenate([q.nodes, X3.reshape(-1, 3)])
    ids = len(q.nodes) + np.arange(X3.shape[0] * 64).reshape(-1, 64)
    spec = dict(q.as_dict())
    spec["nodes"] = nodes
    spec["maps"] = {"hex": (3, ids)}
    m3 = FRMesh(spec, p)
    sc = np.abs(m2.S_u["hex"]).max()
    assert np.abs(m3.S_u["hex"] - m2.S_u["hex"]).max() < 1e-13 * sc
    assert np.abs(m3.detJ["hex"] - m2.detJ["hex"]).max() < 1e-13 * np.abs(m2.detJ["hex"]).max()
    assert np.abs(m3.upts_x["hex"] - m2.upts_x["hex"]).max() < 1e-14


# ------------------------------------------------- cubic prisms, tetrahedra
def _monomials(kind, x):
    """Values (npts, nm) and gradients (3, npts, nm) of the monomial basis of
    the cubic map's space: x^a y^b z^c with a + b + c <= 3 (tetrahedra),
    a + b <= 3 and c <= 3 (prisms)."""
    ex = [(a, b, c) for a in range(4) for b in range(4) for c in range(4)
          if (a + b + c <= 3 if kind == "tet" else a + b <= 3)]

    def pw(v, k):
        return v ** k if k > 0 else np.ones_like(v)

    def dpw(v, k):
        return k * v ** (k - 1) if k > 0 else np.zeros_like(v)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    val = np.stack([pw(X, a) * pw(Y, b) * pw(Z, c) for a, b, c in ex], axis=1)
    grad = np.stack([np.stack([dpw(X, a) * pw(Y, b) * pw(Z, c) for a, b, c in ex], axis=1),
                     np.stack([pw(X, a) * dpw(Y, b) * pw(Z, c) for a, b, c in ex], axis=1),
                     np.stack([pw(X, a) * pw(Y, b) * dpw(Z, c) for a, b, c in ex], axis=1)])
    return val, grad


@pytest.mark.parametrize("kind,nmap", [("pri", 40), ("tet", 20)])
def test_cubic_simplex_map_basis_is_the_lagrange_basis_of_its_space(kind, nmap):
    """The cubic map's shape functions are 1 at their own node and 0 at the
    others, and they reproduce every polynomial of the space (values and
    gradients, against the monomials' own derivatives) at random points."""
    from oracle.elements import element
    el = element(kind, 2)
    nodes = el.q3_nodes()
    assert nodes.shape == (nmap, 3)
    assert np.abs(el.q3_shape(nodes) - np.eye(nmap)).max() < 1e-13
    from frinputs.meshes import _Q3_REF                 # the inputs' node order
    assert np.abs(_Q3_REF[kind] - nodes).max() < 1e-15
    rng = np.random.default_rng(11)
    lam = rng.dirichlet(np.ones(4), 64)
    if kind == "tet":
        x = -1 + 2 * lam[:, 1:]
    else:
        x = np.column_stack([-1 + 2 * lam[:, 1], -1 + 2 * lam[:, 2], rng.uniform(-1, 1, 64)])
    mv, mg = _monomials(kind, x)
    nv, _ = _monomials(kind, nodes)
    assert mv.shape[1] == nmap                      # the space's dimension
    c = rng.normal(size=(nmap, 2))
    f_nodes = nv @ c
    assert np.abs(el.q3_shape(x) @ f_nodes - mv @ c).max() < 1e-12
    for j in range(3):
        assert np.abs(el.q3_dshape(x)[j] @ f_nodes - mg[j] @ c).max() < 1e-11


def _cubic_spec(spec, kind, X3):
    nodes = np.concatenate([spec.nodes, X3.reshape(-1, 3)])
    ids = len(spec.nodes) + np.arange(X3.shape[0] * X3.shape[1]).reshape(X3.shape[:2])
    d = dict(spec.as_dict())
    d["nodes"] = nodes
    d["maps"] = {kind: (3, ids)}
    return d


@pytest.mark.parametrize("kind", ["pri", "tet"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_curl_metric_of_straight_simplices_written_as_cubic_maps(kind, p):
    """Straight prisms and tetrahedra written as cubic maps: the curl form
    equals the map's analytic metric (to 5e-13: the cubic basis, with
    coefficients up to 27, and the products X_l dX_m round a few times more
    than the quadratic one)."""
    lin = mixed_box(n=2, x_pri=0.0 if kind == "pri" else 1.0, x_tet=1.0 if kind == "pri" else 0.0,
                    perturb=0.05)
    ml = FRMesh(lin.as_dict(), p)
    el = ml.el[kind]
    mc = FRMesh(_cubic_spec(lin, kind, el.map_points(lin.nodes[lin.elements[kind]],
                                                     el.q3_nodes())), p)
    scale = np.abs(ml.S_u[kind]).max()
    assert np.abs(mc.S_u[kind] - ml.S_u[kind]).max() < 5e-13 * scale
    assert np.abs(mc.fmag[kind] - ml.fmag[kind]).max() < 5e-13 * scale
    assert np.abs(mc.detJ[kind] - ml.detJ[kind]).max() < 1e-13 * np.abs(ml.detJ[kind]).max()


@pytest.mark.parametrize("kind", ["pri", "tet"])
@pytest.mark.parametrize("p", [2, 4])
def test_quadratic_simplices_written_as_cubic_give_the_same_metric(kind, p):
    q = _jittered(curved_mixed_box(n=2, x_pri=0.0 if kind == "pri" else 1.0,
                                   x_tet=1.0 if kind == "pri" else 0.0), 2)
    keep = {kind: q.elements[kind]}
    q.elements = keep
    q.maps = {kind: q.maps[kind]}
    q.bfaces = []
    q.periodic = [np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])]
    m2 = FRMesh(q.as_dict(), p)
    el = m2.el[kind]
    X2 = q.nodes[q.maps[kind][1]]
    X3 = np.einsum("pv,evk->epk", el.q2_shape(el.q3_nodes()), X2)
    m3 = FRMesh(_cubic_spec(q, kind, X3), p)
    sc = np.abs(m2.S_u[kind]).max()
    assert np.abs(m3.S_u[kind] - m2.S_u[kind]).max() < 1e-13 * sc
    assert np.abs(m3.fmag[kind] - m2.fmag[kind]).max() < 1e-13 * sc
    assert np.abs(m3.detJ[kind] - m2.detJ[kind]).max() < 1e-13 * np.abs(m2.detJ[kind]).max()
    assert np.abs(m3.upts_x[kind] - m2.upts_x[kind]).max() < 1e-14


def _cubic_mixed(**kw):
    """Jittered cubic maps on the mixed box (a = 0.05 h / 3: the Kuhn
    tetrahedra's cubic maps invert near a = 0.1 h / 3)."""
    return _jittered(curved_mixed_box(n=3, order=3, **kw), 3, frac=0.05, order=3)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_cubic_mixed_mesh_free_stream_and_divergence(p):
    """64-node hexahedra, 40-node prisms and 20-node tetrahedra with generic
    maps: free stream kept, discretely divergence-free metrics."""
    m = FRMesh(_cubic_mixed().as_dict(), p)
    assert m.types == ["hex", "pri", "tet"]
    assert _free_stream_residual(m, "ns") < 1e-10
    for t in ("pri", "tet"):
        el, S = m.el[t], m.S_u[t]
        for n in range(3):
            div = sum(np.einsum("pq,eq->ep", el.D[i], S[:, :, i, n]) for i in range(3))
            assert np.abs(div).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("layout", [(0.0, 1.0), (0.0, 0.0), (0.5, 1.0)])
def test_cubic_mixed_mesh_conservation(layout):
    """All prisms, all tetrahedra, hexahedra | prisms; cubic maps, periodic:
    the interface fluxes of both sides of every curved face cancel."""
    m = FRMesh(_cubic_mixed(x_pri=layout[0], x_tet=layout[1], periodic_x=True).as_dict(), 3)
    u = {t: ics.flow3d(m.upts_x[t].reshape(-1, 3)).reshape(m.ne[t], -1, 5) for t in m.types}
    R = FRSystem(m, "ns", mu=0.02).rhs(u)
    tot = sum(np.einsum("q,eq,eqk->k", m.el[t].W, m.detJ[t], R[t]) for t in m.types)
    scale = sum(np.einsum("q,eq,eqk->k", m.el[t].W, m.detJ[t], np.abs(R[t])) for t in m.types)
    assert np.all(np.abs(tot) < 1e-13 * scale.max()), tot / scale.max()


def test_cubic_simplices_pointwise_metric_loses_free_stream():
    spec = _cubic_mixed()
    orig = omesh.curl_metric
    omesh.curl_metric = lambda el, Xm, pts, order=2: _pointwise3(el, Xm, pts)
    try:
        mx = FRMesh(spec.as_dict(), 2)
    finally:
        omesh.curl_metric = orig
    assert _free_stream_residual(mx) > 1e-2
    assert _free_stream_residual(FRMesh(spec.as_dict(), 2)) < 1e-10
