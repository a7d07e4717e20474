"""GPU parity of the tensor-core (tcgen05, split TF32) prism and tetrahedron
kernels: the FP32 family FR_VARIANT_TENSOR against the FP64 oracle and
against the CUDA-core dense kernels.

Tolerances are those of the FP32 mode (see test_gpu_parity): 2e-5 on a
right-hand side and 1e-6 on a solution after a few steps.  The three-term
TF32 product (A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation) drops
only A_lo B_lo, of relative size 2^-22 per term, so the tensor-core result
sits at the FP32 rounding level of the CUDA-core result.

The meshes are mixed_box layouts: 3^3 cells give 18 prisms and 54
tetrahedra, which leave a ragged last tile for every tile size the kernels
use (4, 8 or 16 elements); 16^3 cells give more tiles than resident CTAs, so
the persistent loop runs several times per CTA.
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
    # every conserved variable's right-hand side O(1): a per-variable
    # relative norm then measures each one against a comparable scale
    return ics.flow3d(x)


def _pair(spec, p, physics, bcs=BCS):
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, physics, gamma=1.4, mu=0.02, pr=0.71, bcs=bcs)
    g = fr.FRMesh(spec, p, physics=physics, gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=bcs, precision="fp32")
    g.set_variant("tensor")
    return o, osys, g


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_tensor_rhs_against_oracle(p, physics):
    """Bare right-hand side (hexahedra sum-factorised, prisms and tetrahedra
    on the tensor cores where the order has that form) against the oracle."""
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o, osys, g = _pair(spec, p, physics)
    g.set_solution(lib_state(g, _ic))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _ic)))
    assert err.max() < 2e-5, err


@pytest.mark.parametrize("scheme", ["rk4", "rk45"])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_tensor_rk_steps_against_oracle(scheme, physics):
    """RK stages through the tensor-core epilogue (register update and the
    next stage's u_f = M0 u computed by an MMA)."""
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o, osys, g = _pair(spec, 3, physics)
    g.set_solution(lib_state(g, _ic))
    u = oracle_state(o, _ic)
    dt = 2e-4
    for _ in range(3):
        u = rk.step(osys.rhs, u, dt, scheme)
    g.rk_step(scheme, dt, 3)
    err = rel_l2(g.get_solution(), u)
    assert err.max() < 1e-6, err


@pytest.mark.parametrize("layout", [(0.0, 0.0), (0.0, 1.0)])
def test_tensor_prism_or_tet_only_periodic(layout):
    spec = mixed_box(n=3, x_pri=layout[0], x_tet=layout[1], perturb=0.05,
                     periodic_x=True)
    o, osys, g = _pair(spec, 3, "ns", bcs=None)
    g.set_solution(lib_state(g, _ic))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _ic)))
    # every element of these meshes goes through the split-TF32 products:
    # each operator product drops the lo x lo term (2^-22 relative per
    # term, K = 20..68 terms) on top of FP32 rounding, and the momentum
    # right-hand sides, measured against their own norms, are ~1/15 of the
    # energy's, whose O(1/(gamma Ma^2)) fluxes set the absolute rounding
    assert err.max() < 4e-5, err


@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_tensor_equals_cuda_core_on_many_tiles(physics):
    """16^3 cells (2730 prisms, 8190 tetrahedra): the persistent tensor-core
    kernels loop over several tiles per CTA; their RK steps agree with the
    CUDA-core dense kernels to FP32 rounding."""
    spec = mixed_box(n=16, x_pri=0.34, x_tet=0.67, perturb=0.05)
    out = {}
    for variant in ("sumfact", "tensor"):
        g = fr.FRMesh(spec, 3, physics=physics, gamma=1.4, mu=0.02,
                      prandtl=0.71, bcs=BCS, precision="fp32")
        g.set_variant(variant)
        g.set_solution(lib_state(g, _ic))
        r = g.rhs()
        g.rk_step("rk45", 1e-4, 2)
        out[variant] = (r, g.get_solution())
        assert g.tuning()[0] == variant
    assert rel_l2_rhs(out["tensor"][0], out["sumfact"][0]).max() < 2e-5
    assert rel_l2(out["tensor"][1], out["sumfact"][1]).max() < 1e-6


def test_autotuner_considers_the_tensor_family():
    spec = mixed_box(n=6, x_pri=0.34, x_tet=0.67, perturb=0.05)
    g = fr.FRMesh(spec, 3, physics="ns", gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=BCS, precision="fp32")
    g.set_solution(lib_state(g, _ic))
    g.rk_step("rk45", 1e-4, 1)
    active, ms = g.tuning()
    assert "tensor" in ms and active in ms
    assert ms[active] == min(ms.values())
