"""Gauss-Lobatto hexahedra on the GPU (Section 3.1, "Matrix
multiplications", last paragraph: flux points that are solution points make
the interpolation of Eq. (disu) a gather) against the FP64 oracle with the
same point family.  Tolerances as in test_gpu_parity: FP64 right-hand sides
1e-12 per conserved variable, FP64 solutions 1e-12, FP32 solutions 1e-6."""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, curved_box_hex, ics
from frtest import lib_state, oracle_state, rel_l2, rel_l2_rhs
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _pair(spec, p, physics, precision="fp64", variant=None):
    o = OracleMesh(spec.as_dict(), p, family="gll")
    osys = FRSystem(o, physics, gamma=1.4, mu=0.02, pr=0.71)
    g = fr.FRMesh(spec, p, physics=physics, mu=0.02, prandtl=0.71,
                  precision=precision, family="gll")
    if variant:
        g.set_variant(variant)
    assert np.abs(g.points("hex") - o.upts_x["hex"]).max() < 1e-14
    return o, osys, g


@pytest.mark.parametrize("variant", ["sumfact", "dense"])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_gll_rhs_fp64(p, physics, variant):
    spec = box_hex((3, 3, 2), perturb=0.1)
    o, osys, g = _pair(spec, p, physics, variant=variant)
    g.set_solution(lib_state(g, ics.flow3d))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, ics.flow3d)))
    assert err.max() < 1e-12, err


def test_gll_curved_rhs_fp64():
    spec = curved_box_hex((3, 2, 2))
    o, osys, g = _pair(spec, 3, "ns")
    g.set_solution(lib_state(g, ics.flow3d))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, ics.flow3d)))
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-6),
                                           ("mixed", 1e-6)])
def test_gll_rk45_steps(precision, tol):
    spec = box_hex((3, 3, 2), perturb=0.1)
    o, osys, g = _pair(spec, 3, "ns", precision=precision)
    g.set_solution(lib_state(g, ics.flow3d))
    u = oracle_state(o, ics.flow3d)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    err = rel_l2(g.get_solution(), u)
    assert err.max() < tol, err


def test_gll_vertex_metric_family_fp32():
    spec = box_hex((3, 3, 2), perturb=0.1)
    o, osys, g = _pair(spec, 3, "ns", precision="fp32", variant="sumfact_vertex")
    g.set_solution(lib_state(g, ics.flow3d))
    u = oracle_state(o, ics.flow3d)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    assert rel_l2(g.get_solution(), u).max() < 1e-6


def test_gll_freestream_full_size():
    """A uniform state on 32^3 perturbed Gauss-Lobatto hexahedra, p=3."""
    spec = box_hex((32, 32, 32), hi=(2 * np.pi,) * 3, perturb=0.1)
    g = fr.FRMesh(spec, 3, physics="ns", mu=1 / 1600, prandtl=0.71, family="gll")
    g.set_solution(lib_state(g, ics.uniform))
    assert np.abs(g.rhs()["hex"]).max() < 1e-10
