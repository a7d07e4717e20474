"""Pins for the oracle's curved (quadratic) hexahedra and their conservative
metric ("Curved Elements", Section 3.4): the curl form keeps a uniform flow
uniform on curved grids where the pointwise cross-product metric does not
(the comparison the paper draws in its free-stream figure)."""
import numpy as np
import pytest

from frinputs import box_hex, curved_box_hex, ics
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


def _cross_product_metric(m, spec):
    """Replace the mesh's metric by the map's pointwise cross-product one."""
    el = m.el["hex"]
    Xm = spec.nodes[spec.maps["hex"][1]]

    def cross(x):
        a = np.einsum("jpv,evk->epjk", el.q2_dshape(x), Xm)
        return np.stack([np.cross(a[:, :, 1], a[:, :, 2]),
                         np.cross(a[:, :, 2], a[:, :, 0]),
                         np.cross(a[:, :, 0], a[:, :, 1])], axis=2)
    m.S_u["hex"] = cross(el.upts)
    nv = np.einsum("epij,pi->epj", cross(el.fpts), el.fpts_norm)
    mag = np.linalg.norm(nv, axis=2)
    m.fmag["hex"] = mag
    m.fnorm["hex"] = nv / mag[:, :, None]


@pytest.mark.parametrize("p", [2, 3])
def test_curl_metric_is_discretely_divergence_free(p):
    m = FRMesh(curved_box_hex((3, 3, 3)).as_dict(), p)
    el, S = m.el["hex"], m.S_u["hex"]
    for n in range(3):
        div = sum(np.einsum("pq,eq->ep", el.D[i], S[:, :, i, n]) for i in range(3))
        assert np.abs(div).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("p", [2, 3])
def test_free_stream_kept_by_conservative_metric_not_by_cross_product(p):
    spec = curved_box_hex((3, 3, 3))
    m = FRMesh(spec.as_dict(), p)
    R = FRSystem(m, "euler").rhs(_uniform(m))["hex"]
    assert np.abs(R).max() < 1e-10          # residual scale ~1e2
    _cross_product_metric(m, spec)
    Rx = FRSystem(m, "euler").rhs(_uniform(m))["hex"]
    assert np.abs(Rx).max() > 1e-3


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
