"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
and its host-side set-up (points, operators, metrics, interface pairing,
mesh validation) agrees with the independently written oracle.  No GPU is
touched: handles are created with device = -1 (host-only)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, curved_box_hex, curved_mixed_box, mixed_box
from oracle.mesh import FRMesh as OracleMesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s+(fr_\w+)\s*\(",
                                txt, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(fr.build())
    names = _declared()
    assert "fr_rhs" in names and "fr_rk_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_compute_calls_refuse_host_only_handles():
    g = fr.FRMesh(box_hex((2, 2, 2)), 2, device=-1)
    with pytest.raises(fr.FRError) as e:
        g.rhs()
    assert e.value.name == "FR_EINVAL"
    st = g.stats()
    assert st["rhs_calls"] == 0 and st["ms_device"] == 0.0


def test_rhs_rejects_a_non_finite_time():
    lib = fr.load()
    g = fr.FRMesh(box_hex((2, 2, 2)), 2, device=-1)
    assert lib.fr_rhs(g._h, float("nan"), None, None) == -1
    assert lib.fr_stats(None, None, 0) == -1


SPECS = {
    "hex": lambda: box_hex((3, 2, 2), perturb=0.1),
    "hex-gll": lambda: box_hex((3, 2, 2), perturb=0.1),
    "curved-gll": lambda: curved_box_hex((3, 2, 2)),
    "curved-mixed": lambda: curved_mixed_box(n=3),
    "curved-cubic": lambda: curved_box_hex((3, 2, 2), order=3),
    "curved-mixed-cubic": lambda: curved_mixed_box(n=3, order=3),
    "mixed": lambda: mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05),
    "curved": lambda: curved_box_hex((3, 2, 2)),
}


@pytest.mark.parametrize("name", list(SPECS))
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_host_setup_matches_oracle(name, p):
    spec = SPECS[name]()
    fam = "gll" if name.endswith("-gll") else "gl"
    bcs = {k: ("state", 1.0, 0.0, 0.0, 0.0, 1.0) for k in range(6)}
    g = fr.FRMesh(spec, p, bcs=bcs, device=-1, family=fam)
    o = OracleMesh(spec.as_dict(), p, family=fam)
    assert g.types == o.types
    for t in g.types:
        el = o.el[t]
        assert np.abs(g.operator(t, "upts") - el.upts).max() < 1e-15
        assert np.abs(g.operator(t, "fpts") - el.fpts).max() < 1e-15
        assert np.abs(g.operator(t, "M0") - el.M0).max() < 1e-13
        for d in range(3):
            assert np.abs(g.operator(t, "D")[d] - el.D[d]).max() < 1e-13
        assert np.abs(g.operator(t, "LIFT") - el.LIFT).max() < 5e-13
        assert np.abs(g.operator(t, "W") - el.W).max() < 1e-13
        assert np.abs(g.points(t) - o.upts_x[t]).max() < 1e-14
        S, rj = g.metrics(t)
        So = o.S_u[t].reshape(o.ne[t], -1, 9).transpose(0, 2, 1)
        # the host library and the oracle sum in different orders: 1e-13 of
        # the metric's scale; 5e-13 for cubic simplex maps, whose curl form
        # cancels terms X_l dX_m some 10x larger than S, built from basis
        # coefficients up to 27
        tol = 5e-13 if name == "curved-mixed-cubic" else 1e-13
        assert np.abs(S - So).max() < tol * np.abs(So).max()
        assert np.abs(rj * o.detJ[t] - 1).max() < 1e-13
    npair, nb = g.pair_counts()
    assert npair == len(o.pair_l) and nb == len(o.bnd_g)


def test_gll_family_rejects_prisms():
    with pytest.raises(fr.FRError) as e:
        fr.FRMesh(mixed_box(n=3, x_pri=0.34, x_tet=0.67), 2, device=-1, family="gll")
    assert e.value.name == "FR_EINVAL"


def test_nonconforming_mesh_is_rejected():
    spec = box_hex((2, 2, 2), periodic=(0, 1))
    spec.bfaces = []
    with pytest.raises(fr.FRError) as e:
        fr.FRMesh(spec, 2, device=-1)
    assert e.value.name == "FR_EMESH"


def test_inverted_element_is_rejected():
    spec = box_hex((2, 2, 2))
    conn = spec.elements["hex"].copy()
    conn[0] = conn[0][[4, 5, 6, 7, 0, 1, 2, 3]]     # mirrored: det J < 0
    spec.elements = {"hex": conn}
    with pytest.raises(fr.FRError) as e:
        fr.FRMesh(spec, 2, device=-1)
    assert e.value.name == "FR_EMESH"


def test_bad_arguments():
    spec = box_hex((2, 2, 2))
    with pytest.raises(fr.FRError):
        fr.FRMesh(spec, 9, device=-1)
    with pytest.raises(fr.FRError):
        fr.FRMesh(spec, 2, gamma=1.0, device=-1)
    spec2 = box_hex((2, 2, 2), periodic=(0, 1))
    # z faces listed with a tag that has no boundary condition
    with pytest.raises(fr.FRError):
        fr.FRMesh(spec2, 2, device=-1)


def test_single_element_periodic_with_itself():
    spec = box_hex((1, 1, 1))
    g = fr.FRMesh(spec, 2, device=-1)
    o = OracleMesh(spec.as_dict(), 2)
    assert g.pair_counts() == (len(o.pair_l), 0)


def test_curved_maps_are_validated():
    """A quadratic map whose corner nodes are not the element's vertices, a
    node id out of range, or a quadratic map on a non-hexahedron is refused
    at creation."""
    spec = curved_box_hex((2, 2, 2))
    order, mconn = spec.maps["hex"]
    bad = mconn.copy()
    bad[0, [0, 2]] = bad[0, [2, 0]]
    spec.maps["hex"] = (order, bad)
    with pytest.raises(fr.FRError):
        fr.FRMesh(spec, 2, device=-1)
    bad = mconn.copy()
    bad[1, 13] = len(spec.nodes)
    spec.maps["hex"] = (order, bad)
    with pytest.raises(fr.FRError):
        fr.FRMesh(spec, 2, device=-1)
    m = mixed_box(n=2, x_pri=0.5, x_tet=1.0)
    m.maps = {"pri": (2, np.zeros((len(m.elements["pri"]), 27), np.int64))}
    with pytest.raises(fr.FRError):
        fr.FRMesh(m, 2, device=-1)


@pytest.mark.parametrize("name", ["hex", "mixed", "curved"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_antialias_operators_match_oracle(name, p):
    """Anti-aliasing rule (points, weights), interpolation B and projection
    P of every type against the oracle's.  The two enumerate the rule's
    points in different orders: points are matched by coordinates."""
    spec = SPECS[name]()
    bcs = {k: ("extrap",) for k in range(6)}
    g = fr.FRMesh(spec, p, bcs=bcs, device=-1)
    o = OracleMesh(spec.as_dict(), p)
    qdeg = 3 * p
    g.set_antialias(qdeg)
    for t in g.types:
        xo, wo, Bo, Po = o.el[t].aa_operators(qdeg)
        x = g.operator(t, "aa_qpts")
        assert x.shape == xo.shape
        d = np.linalg.norm(x[:, None, :] - xo[None, :, :], axis=2)
        perm = d.argmin(axis=1)
        assert np.abs(d[np.arange(len(x)), perm]).max() < 1e-14
        assert len(set(perm.tolist())) == len(x)
        assert np.abs(g.operator(t, "aa_qwts") - wo[perm]).max() < 1e-15
        assert np.abs(g.operator(t, "aa_B") - Bo[perm]).max() < 1e-13
        assert np.abs(g.operator(t, "aa_P") - Po[:, perm]).max() < 1e-13
    g.set_antialias(0)
    with pytest.raises(fr.FRError):
        g.operator(g.types[0], "aa_B")


@pytest.mark.parametrize("name", ["hex", "mixed", "curved"])
def test_interface_orientation_matches_oracle(name):
    """The library orients every interface by the rule the oracle applies
    independently (lower global element on the "-" side): the multisets of
    (left element, right element) pairs agree."""
    spec = SPECS[name]()
    bcs = {k: ("extrap",) for k in range(6)}
    g = fr.FRMesh(spec, 2, bcs=bcs, device=-1)
    o = OracleMesh(spec.as_dict(), 2)
    left, right = g.interfaces()
    assert np.all(left <= right)
    eoff, n = {}, 0
    for t in o.types:
        eoff[t] = n
        n += o.ne[t]

    def elem(gidx):
        out = np.empty(len(gidx), np.int64)
        for t in o.types:
            lo = o.foff[t]
            hi = lo + o.ne[t] * o.el[t].nfpts
            sel = (gidx >= lo) & (gidx < hi)
            out[sel] = eoff[t] + (gidx[sel] - lo) // o.el[t].nfpts
        return out
    ol, orr = elem(o.pair_l), elem(o.pair_r)
    lib = sorted(zip(left.tolist(), right.tolist()))
    ora = sorted(zip(ol.tolist(), orr.tolist()))
    assert lib == ora


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_prism_operators_factor_into_triangle_and_line(p):
    """The prism's operators as the library builds them have the structure
    its structured kernels read: D_xi and D_eta act within a level of the
    triangle x line points (the same block on every level), D_zeta along a
    line (the same 1D operator for every triangle point), and M0 / LIFT rows
    touch few points (the line through a triangle-face point, the edge of a
    level for a quadrilateral face).  Checked here on the host from the
    library's own dense operators, against the point order z * NT + t."""
    bcs = {k: ("state", 1.0, 0.2, 0.0, 0.0, 5.0) for k in range(4)}
    g = fr.FRMesh(mixed_box(n=2, x_pri=0.0, x_tet=1.1), p, bcs=bcs, device=-1)
    D = g.operator("pri", "D")
    M0 = g.operator("pri", "M0")
    L = g.operator("pri", "LIFT")
    nt, nl = (p + 1) * (p + 2) // 2, p + 1
    nu = nt * nl
    assert D.shape == (3, nu, nu)
    tol = 1e-12 * np.abs(D).max()
    lev = np.arange(nu) // nt
    tri = np.arange(nu) % nt
    same_level = lev[:, None] == lev[None, :]
    same_line = tri[:, None] == tri[None, :]
    for d in (0, 1):
        assert np.abs(D[d][~same_level]).max() <= tol
        blk = D[d][:nt, :nt]
        for z in range(nl):
            assert np.abs(D[d][z * nt:(z + 1) * nt, z * nt:(z + 1) * nt] - blk).max() <= tol
    assert np.abs(D[2][~same_line]).max() <= tol
    line = D[2][::nt, ::nt]
    for t in range(nt):
        assert np.abs(D[2][t::nt, t::nt] - line).max() <= tol
    nz_m0 = (np.abs(M0) > 1e-12 * np.abs(M0).max()).sum(axis=1)
    nz_l = (np.abs(L) > 1e-12 * np.abs(L).max()).sum(axis=1)
    if p <= 3:
        # the triangle-face flux points are the solution points' triangle
        # points: every M0 row is the p + 1 points of a line or an edge,
        # within the kernels' bounds (16 per M0 row, 64 per LIFT row)
        assert nz_m0.max() == nl and nz_l.max() <= 64
    else:
        # at p = 4 the triangle-face points differ from the solution
        # triangle points: those rows are dense (the library keeps the dense
        # kernels for this order)
        assert nz_m0.max() == nu


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tetrahedron_flux_points_are_solution_points(p):
    """Every flux point of the library's tetrahedron is one of its solution
    points (its M0 row has a single nonzero, 1): the CUDA-core kernels take
    the interpolation to the flux points as a gather."""
    bcs = {k: ("state", 1.0, 0.2, 0.0, 0.0, 5.0) for k in range(4)}
    g = fr.FRMesh(mixed_box(n=2, x_pri=0.34, x_tet=0.67), p, bcs=bcs, device=-1)
    M0 = g.operator("tet", "M0")
    nz = np.abs(M0) > 1e-12 * np.abs(M0).max()
    assert np.all(nz.sum(axis=1) == 1)
    assert np.allclose(M0[nz], 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("p", [2, 3])
def test_library_curl_metrics_are_discretely_divergence_free(order, p):
    """The library's own curved metrics, with its own derivative operators
    (no oracle): sum_i D_i S[i][n] = 0 at the solution points of every type,
    for quadratic and cubic maps (S in the element's solution space)."""
    g = fr.FRMesh(curved_mixed_box(n=3, order=order), p, device=-1,
                  bcs={k: ("state", 1.0, 0.0, 0.0, 0.0, 1.0) for k in range(6)})
    for t in g.types:
        S, _ = g.metrics(t)                    # (ne, 9, nu), row i*3 + n
        D = g.operator(t, "D")                 # (3, nu, nu)
        scale = np.abs(S).max()
        for n in range(3):
            div = sum(np.einsum("pq,eq->ep", D[i], S[:, 3 * i + n, :]) for i in range(3))
            assert np.abs(div).max() < 1e-12 * scale, (t, n, np.abs(div).max() / scale)
