"""GPU parity of the structured prism kernels (k_grad_pri, k_vol_pri): the
triangle x line factorisation of the prism's derivative operators and the
nonzeros of its interpolation and lift (Section 3.1, "Matrix
multiplications").  Prisms run them in every family but the dense one at
orders 1-3 (at p = 4 the triangle-face interpolation is dense and the dense
kernels stay).  Tetrahedra take their interpolation to the flux points as a
gather in the same families (their flux points are solution points).

Tolerances are those of the other parity tests: FP64 1e-12 relative L2 per
conserved variable against the oracle, and the structured and dense FP64
kernels agree to 1e-13 (the same products without the zero terms); FP32
2e-5 on a right-hand side, 1e-6 on a solution after a few steps.

Meshes: mixed_box layouts; 3^3 cells give 18 prisms (a ragged last group
of the 6 (p=3) to 42 (p=1) elements a CTA takes), 12^3 cells more groups
than resident CTAs, so the persistent loop runs several times per CTA.
"""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import ics, mixed_box
from frtest import lib_state, oracle_state, rel_l2, rel_l2_rhs
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh

pytestmark = pytest.mark.gpu

BCS = {0: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       1: ("extrap",),
       2: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       3: ("extrap",)}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _ic(x):
    return ics.flow3d(x)


def _mesh(spec, p, physics, precision, variant):
    g = fr.FRMesh(spec, p, physics=physics, gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=BCS, precision=precision)
    g.set_variant(variant)
    return g


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_structured_prism_rhs_fp64_against_oracle(p, physics):
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, physics, gamma=1.4, mu=0.02, pr=0.71, bcs=BCS)
    g = _mesh(spec, p, physics, "fp64", "sumfact")
    g.set_solution(lib_state(g, _ic))
    r = g.rhs()
    assert g.schedule()["pri"]["structured"]
    err = rel_l2_rhs(r, osys.rhs(oracle_state(o, _ic)))
    assert err.max() < 1e-12, err
    # the dense kernels on the same state: the same products plus zeros
    h = _mesh(spec, p, physics, "fp64", "dense")
    h.set_solution(lib_state(h, _ic))
    rd = h.rhs()
    assert not h.schedule()["pri"]["structured"]
    err = rel_l2_rhs(r, rd)
    assert err.max() < 1e-13, err


def test_order_4_prisms_keep_the_dense_kernels():
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    g = _mesh(spec, 4, "ns", "fp64", "sumfact")
    g.set_solution(lib_state(g, _ic))
    g.rhs()
    assert not g.schedule()["pri"]["structured"]
    assert g.schedule()["hex"]["structured"]


@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_structured_prism_fp32_against_oracle(physics):
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o = OracleMesh(spec.as_dict(), 3)
    osys = FRSystem(o, physics, gamma=1.4, mu=0.02, pr=0.71, bcs=BCS)
    g = _mesh(spec, 3, physics, "fp32", "sumfact")
    g.set_solution(lib_state(g, _ic))
    r = g.rhs()
    assert g.schedule()["pri"]["structured"]
    err = rel_l2_rhs(r, osys.rhs(oracle_state(o, _ic)))
    assert err.max() < 2e-5, err


@pytest.mark.parametrize("scheme", ["rk4", "rk45"])
def test_structured_prism_rk_steps_fp64(scheme):
    """RK stages through the structured kernels' epilogue and next-stage
    interpolation, on a mesh with more prism groups than resident CTAs."""
    spec = mixed_box(n=12, x_pri=0.2, x_tet=0.9, perturb=0.05)
    g = _mesh(spec, 3, "ns", "fp64", "sumfact")
    h = _mesh(spec, 3, "ns", "fp64", "dense")
    for m in (g, h):
        m.set_solution(lib_state(m, _ic))
        m.rk_step(scheme, 2e-4, 3)
    assert g.schedule()["pri"]["structured"]
    err = rel_l2(g.get_solution(), h.get_solution())
    assert err.max() < 1e-13, err


def test_structured_prism_rk_steps_against_oracle():
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o = OracleMesh(spec.as_dict(), 2)
    osys = FRSystem(o, "ns", gamma=1.4, mu=0.02, pr=0.71, bcs=BCS)
    g = _mesh(spec, 2, "ns", "fp64", "sumfact")
    g.set_solution(lib_state(g, _ic))
    u = oracle_state(o, _ic)
    dt = 2e-4
    for _ in range(3):
        u = rk.step(osys.rhs, u, dt, "rk45")
    g.rk_step("rk45", dt, 3)
    err = rel_l2(g.get_solution(), u)
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("p", [2, 3, 4])
def test_tetrahedron_gather_matches_dense_and_oracle(p):
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, "ns", gamma=1.4, mu=0.02, pr=0.71, bcs=BCS)
    g = _mesh(spec, p, "ns", "fp64", "sumfact")
    g.set_solution(lib_state(g, _ic))
    r = g.rhs()
    assert g.schedule()["tet"]["structured"]
    err = rel_l2_rhs(r, osys.rhs(oracle_state(o, _ic)))
    assert err.max() < 1e-12, err
    h = _mesh(spec, p, "ns", "fp64", "dense")
    h.set_solution(lib_state(h, _ic))
    rd = h.rhs()  # the family takes effect at the first evaluation
    assert not h.schedule()["tet"]["structured"]
    err = rel_l2_rhs(r, rd)
    assert err.max() < 1e-13, err
