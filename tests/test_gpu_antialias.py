"""GPU parity of the anti-aliased flux (Section 3.2, "Anti-aliasing":
quadrature-point flux, least-squares projection onto the solution space)
against the oracle's FRSystem(antialias=qdeg).

Tolerances as for collocation: FP64 right-hand sides 1e-12 relative L2
(5e-12 at p = 4), FP64 solutions 1e-12, FP32 solutions 1e-6, mixed form
1e-6 against the FP64 oracle after two steps.
"""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, curved_box_hex, ics, mixed_box
from frtest import lib_state, oracle_state, rel_l2, rel_l2_rhs
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh

pytestmark = pytest.mark.gpu

BCS = {0: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       1: ("extrap",),
       2: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       3: ("extrap",)}

SPECS = {
    "hex": lambda: box_hex((3, 3, 2), perturb=0.1),
    "mixed": lambda: mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05),
    "curved": lambda: curved_box_hex((3, 3, 2)),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _tgv(x):
    # every conserved variable's right-hand side O(1): a per-variable
    # relative norm then measures each one against a comparable scale
    return ics.flow3d(x)


def _pair(name, p, physics, qdeg, precision="fp64"):
    spec = SPECS[name]()
    bcs = BCS if name == "mixed" else None
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, physics, gamma=1.4, mu=0.02, pr=0.71, bcs=bcs,
                    antialias=qdeg)
    g = fr.FRMesh(spec, p, physics=physics, gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=bcs, precision=precision)
    g.set_antialias(qdeg)
    return o, osys, g


@pytest.mark.parametrize("name", ["hex", "mixed", "curved"])
@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_aa_rhs_fp64(name, p, physics):
    o, osys, g = _pair(name, p, physics, 3 * p)
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < (5e-12 if p == 4 else 1e-12), err


@pytest.mark.parametrize("qdeg", [1, 5, 8, 11])
def test_aa_rule_degrees(qdeg):
    """Rules below, at and above the solution space's degree (qdeg 1 is a
    single point per direction)."""
    o, osys, g = _pair("mixed", 3, "ns", qdeg)
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("variant", ["sumfact", "dense"])
def test_aa_rk_steps_fp64(variant):
    o, osys, g = _pair("hex", 3, "ns", 9)
    g.set_variant(variant)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(3):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 3)
    assert rel_l2(g.get_solution(), u).max() < 1e-12


@pytest.mark.parametrize("name,variant", [("hex", "sumfact"), ("hex", "dense"),
                                          ("hex", "sumfact_vertex"),
                                          ("mixed", "dense"), ("mixed", "tensor"),
                                          ("curved", "sumfact")])
def test_aa_fp32_families(name, variant):
    """FP32 values; the vertex-metric family is replaced by the stored-metric
    one and the tensor family keeps its gradient kernels only."""
    o, osys, g = _pair(name, 3, "ns", 9, precision="fp32")
    g.set_variant(variant)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    assert rel_l2(g.get_solution(), u).max() < 1e-6
    assert g.tuning()[0] != "sumfact_vertex"


def test_aa_mixed_precision():
    o, osys, g = _pair("hex", 3, "ns", 9, precision="mixed")
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    assert rel_l2(g.get_solution(), u).max() < 1e-6


def test_aa_off_restores_collocation_exactly():
    """Switching the projection off gives back the collocated right-hand
    side bit for bit (the graphs are rebuilt both ways)."""
    spec = SPECS["mixed"]()
    kw = dict(physics="ns", mu=0.02, prandtl=0.71, bcs=BCS)
    g = fr.FRMesh(spec, 3, **kw)
    h = fr.FRMesh(spec, 3, **kw)
    for m in (g, h):
        m.set_solution(lib_state(m, _tgv))
    g.set_antialias(9)
    g.rk_step("rk45", 1e-3, 1)
    g.set_antialias(0)
    g.set_solution(lib_state(g, _tgv))
    g.rk_step("rk45", 1e-3, 1)
    h.rk_step("rk45", 1e-3, 1)
    for t in g.types:
        assert np.array_equal(g.get_solution()[t], h.get_solution()[t])


def test_aa_profile_and_tuner():
    spec = box_hex((5, 5, 5), perturb=0.1)
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71, precision="fp32")
    g.set_antialias(9)
    g.set_solution(lib_state(g, _tgv))
    g.rk_step("rk45", 1e-3, 1)
    active, ms = g.tuning()
    assert "sumfact_vertex" not in ms and active in ms
    prof = g.profile_step("rk45", 1e-3)
    assert prof["aa_flux"][1] == 5 and prof["aa_flux"][0] > 0


@pytest.mark.parametrize("qdeg", [7, 9, 11])
def test_aa_fp32_hex_point_counts(qdeg):
    """FP32 hexahedra with 4, 5 and 6 rule points per direction at p = 3
    (the general kernel and both compile-time point counts)."""
    o, osys, g = _pair("hex", 3, "ns", qdeg, precision="fp32")
    g.set_variant("sumfact")
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    assert rel_l2(g.get_solution(), u).max() < 1e-6
