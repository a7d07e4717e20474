"""Boundary states prescribed point by point (FR_BC_PRESCRIBED,
fr_set_bc_state: the outside state u+ of Eq. comm_flux given by the caller
at every boundary flux point) against the oracle's ('prescribed', fn)
condition: FP64 right-hand sides 1e-12 per variable, RK steps in FP64
(1e-12) and FP32 (1e-6), a time-dependent state updated between steps."""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, ics, mixed_box
from frtest import lib_state, oracle_state, rel_l2, rel_l2_rhs
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh

pytestmark = pytest.mark.gpu

P_INF = 1.0 / 1.4 / 0.09


def inflow(x, t=0.0):
    """A smooth, spatially varying inflow state (primitive variables)."""
    return np.column_stack([1.0 + 0.1 * np.sin(6 * x[:, 1] + t),
                            0.4 + 0.05 * np.cos(5 * x[:, 2]),
                            0.1 + 0 * x[:, 0],
                            0.05 * np.sin(4 * x[:, 1] + 3 * x[:, 2]),
                            P_INF * (1 + 0.02 * np.cos(6 * x[:, 2] - t))])


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _bcs(fn):
    return {0: ("prescribed", fn), 1: ("extrap",), 2: ("prescribed", fn), 3: ("extrap",)}


def _pair(spec, p, physics, precision="fp64", fn=inflow):
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, physics, mu=0.02, pr=0.71, bcs=_bcs(fn))
    g = fr.FRMesh(spec, p, physics=physics, mu=0.02, prandtl=0.71, bcs=_bcs(fn),
                  precision=precision)
    return o, osys, g


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_prescribed_rhs_fp64(p, physics):
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o, osys, g = _pair(spec, p, physics)
    g.set_solution(lib_state(g, ics.flow3d))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, ics.flow3d)))
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("precision,variant,tol", [("fp64", "sumfact", 1e-12),
                                                   ("fp32", "sumfact", 1e-6),
                                                   ("fp32", "tensor", 1e-6)])
def test_prescribed_rk_steps(precision, variant, tol):
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o, osys, g = _pair(spec, 3, "ns", precision)
    g.set_variant(variant)
    g.set_solution(lib_state(g, ics.flow3d))
    u = oracle_state(o, ics.flow3d)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 2e-4, "rk45")
    g.rk_step("rk45", 2e-4, 2)
    err = rel_l2(g.get_solution(), u)
    assert err.max() < tol, err


def test_prescribed_time_dependent_state_updated_between_steps():
    spec = box_hex((4, 3, 3), periodic=(1, 2), perturb=0.1)
    bcs = {0: ("prescribed", None), 1: ("extrap",)}
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71, bcs=bcs)
    g.set_solution(lib_state(g, ics.flow3d))
    with pytest.raises(fr.FRError) as e:
        g.rk_step("rk4", 1e-4, 1)           # no state yet
    assert e.value.name == "FR_EINVAL"
    o = OracleMesh(spec.as_dict(), 3)
    u = oracle_state(o, ics.flow3d)
    dt = 1e-4
    for step in range(3):
        t = step * dt
        g.set_bc_state(0, inflow, t=t)
        osys = FRSystem(o, "ns", mu=0.02, pr=0.71,
                        bcs={0: ("prescribed", lambda x, t=t: inflow(x, t)), 1: ("extrap",)})
        u = rk.step(osys.rhs, u, dt, "rk4")
        g.rk_step("rk4", dt, 1)
    assert rel_l2(g.get_solution(), u).max() < 1e-12


def test_constant_prescribed_state_equals_state_condition():
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    const = (1.0, 0.4, 0.1, 0.0, P_INF)

    def fn(x):
        return np.tile(const, (len(x), 1))
    a = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71, bcs=_bcs(fn))
    b = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71,
                  bcs={0: ("state",) + const, 1: ("extrap",), 2: ("state",) + const,
                       3: ("extrap",)})
    for m in (a, b):
        m.set_solution(lib_state(m, ics.flow3d))
    assert rel_l2_rhs(a.rhs(), b.rhs()).max() < 1e-15


def test_prescribed_state_rejects_non_positive_density():
    spec = box_hex((3, 2, 2), periodic=(1, 2))
    g = fr.FRMesh(spec, 2, bcs={0: ("prescribed", None), 1: ("extrap",)})
    with pytest.raises(fr.FRError):
        g.set_bc_state(0, lambda x: np.tile((-1.0, 0, 0, 0, 1.0), (len(x), 1)))
