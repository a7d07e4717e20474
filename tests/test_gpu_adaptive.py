"""GPU parity of adaptive time stepping (Section 3.5: low-storage RK with an
embedded pair, error-controlled step size) against the oracle's
adaptive_step: the same accept / reject decisions and step sizes, and the
same solution.

Tolerances: FP64 solutions 1e-12 (as every FP64 solution test); the
normalised errors and the proposed step sizes agree to 1e-9 relative (the
norm sums ~1e4 squared terms in a different order; the controller's powers
amplify nothing beyond that).  FP32: errors to 1e-3 relative (the estimate
is a difference of nearly equal stage combinations, computed from FP32
states), solutions 1e-6 as the other FP32 solution tests.
"""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, ics, mixed_box
from frtest import lib_state, oracle_state, rel_l2
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
    return ics.taylor_green(2 * np.pi * x, mach=0.3)


def _pair(spec, p, precision, bcs=BCS):
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, "ns", gamma=1.4, mu=0.02, pr=0.71, bcs=bcs)
    g = fr.FRMesh(spec, p, physics="ns", gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=bcs, precision=precision)
    return o, osys, g


def _run_both(o, osys, g, dt0, tol, attempts):
    g.set_solution(lib_state(g, _ic))
    u = oracle_state(o, _ic)
    ctl = fr.AdaptCtl(tol, tol, 1.0, 0)
    st = {"err_prev": 1.0, "rejected": False}
    dg = do = dt0
    seq = []
    for _ in range(attempts):
        okg, errg, dg_next = g.rk_adaptive_step(dg, ctl)
        u, oko, erro, do_next = rk.adaptive_step(osys.rhs, u, do, tol, tol, st)
        seq.append((okg, oko, errg, erro, dg_next, do_next))
        dg, do = dg_next, do_next
    return u, seq


def test_adaptive_fp64_matches_oracle():
    """Mixed hex/prism/tet box: a first step far above the stable size is
    rejected, the controller shrinks it, later steps grow; every decision,
    error and step size matches the oracle."""
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    o, osys, g = _pair(spec, 2, "fp64")
    u, seq = _run_both(o, osys, g, 5e-2, 1e-7, 6)
    assert not seq[0][0], "the oversized first step must be rejected"
    assert any(s[0] for s in seq), "some step must be accepted"
    for okg, oko, errg, erro, dg, do in seq:
        assert okg == oko
        if np.isfinite(erro):
            assert abs(errg - erro) <= 1e-9 * max(erro, 1e-30), (errg, erro)
        assert abs(dg - do) <= 1e-9 * do, (dg, do)
    assert rel_l2(g.get_solution(), u).max() < 1e-12


def test_adaptive_fp32_matches_oracle():
    spec = box_hex((3, 3, 2), perturb=0.1)
    o, osys, g = _pair(spec, 3, "fp32", bcs=None)
    u, seq = _run_both(o, osys, g, 2e-2, 1e-5, 5)
    for okg, oko, errg, erro, dg, do in seq:
        assert okg == oko
        assert abs(errg - erro) <= 1e-3 * erro, (errg, erro)
    assert rel_l2(g.get_solution(), u).max() < 1e-6


def test_rejected_step_restores_the_solution():
    """A step far beyond stability (non-finite or huge error) is rejected,
    the state is unchanged bit for bit, and the next accepted step then
    matches a plain RK45 step of the same size."""
    spec = box_hex((2, 2, 2), perturb=0.1)
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71)
    g.set_solution(lib_state(g, _ic))
    before = g.get_solution()["hex"].copy()
    ctl = fr.AdaptCtl(1e-6, 1e-6, 1.0, 0)
    ok, err, dt_next = g.rk_adaptive_step(50.0, ctl)
    assert not ok and err > 1.0 and dt_next < 50.0 and ctl.after_reject == 1
    assert np.array_equal(g.get_solution()["hex"], before)
    ok, err, _ = g.rk_adaptive_step(1e-4, ctl)
    assert ok
    h = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71)
    h.set_solution(lib_state(h, _ic))
    h.rk_step("rk45", 1e-4, 1)
    assert rel_l2(g.get_solution(), h.get_solution()).max() < 1e-13


def test_integrate_adaptive_reaches_the_end_time():
    spec = box_hex((2, 2, 2), perturb=0.1)
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71, precision="fp32")
    g.set_solution(lib_state(g, _ic))
    log = g.integrate_adaptive(2e-2, 1e-3, 1e-5, 1e-5)
    t_end = [t for t, _, ok, _ in log if ok][-1]
    assert abs(t_end - 2e-2) < 1e-12
    assert sum(ok for _, _, ok, _ in log) >= 2
