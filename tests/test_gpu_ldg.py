"""GPU parity of the LDG viscous coupling (beta-biased common solution and
viscous flux along each interface's orientation, penalty tau) against the
oracle's FRSystem(ldg=(beta, tau)).  The library and the oracle orient
every interface independently by the same rule (lower global element on
the "-" side).  Tolerances as for BR1: FP64 right-hand sides 1e-12, FP32
solutions 1e-6."""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, curved_box_hex, ics, mixed_box
from frtest import lib_state, oracle_state, rel_l2, rel_l2_rhs
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh
from paper_2408_16509_gb300 import partition

pytestmark = pytest.mark.gpu

BCS = {0: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       1: ("extrap",),
       2: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       3: ("extrap",)}
SPECS = {"hex": lambda: box_hex((3, 3, 2), perturb=0.1),
         "mixed": lambda: mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05),
         "curved": lambda: curved_box_hex((3, 3, 2))}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _tgv(x):
    # every conserved variable's right-hand side O(1): a per-variable
    # relative norm then measures each one against a comparable scale
    return ics.flow3d(x)


def _pair(name, p, ldg, precision="fp64"):
    spec = SPECS[name]()
    bcs = BCS if name == "mixed" else None
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, "ns", gamma=1.4, mu=0.02, pr=0.71, bcs=bcs, ldg=ldg)
    g = fr.FRMesh(spec, p, physics="ns", gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=bcs, precision=precision)
    g.set_viscous_scheme(*ldg)
    return o, osys, g


@pytest.mark.parametrize("name", ["hex", "mixed", "curved"])
@pytest.mark.parametrize("ldg", [(0.5, 0.1), (-0.3, 0.05)])
def test_ldg_rhs_fp64(name, ldg):
    o, osys, g = _pair(name, 3, ldg)
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("name,variant", [("hex", "sumfact"), ("hex", "sumfact_vertex"),
                                          ("mixed", "dense"), ("mixed", "tensor")])
def test_ldg_fp32_rk(name, variant):
    o, osys, g = _pair(name, 3, (0.5, 0.1), precision="fp32")
    g.set_variant(variant)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    assert rel_l2(g.get_solution(), u).max() < 1e-6


def test_ldg_groups_penalty_only_and_bias_refused():
    spec = box_hex((4, 4, 3), perturb=0.1)
    kw = dict(physics="ns", mu=0.02, prandtl=0.71)
    whole = fr.FRMesh(spec, 3, **kw)
    whole.set_variant("sumfact")
    whole.set_viscous_scheme(0.0, 0.1)
    u = lib_state(whole, _tgv)
    whole.set_solution(u)
    subs, ids, _ = partition.split(spec, 3)
    members = [fr.FRMesh(s, 3, bcs=partition.exchange_bcs({}), **kw) for s in subs]
    for g, ur in zip(members, partition.scatter(u, ids)):
        g.set_variant("sumfact")
        g.set_viscous_scheme(0.0, 0.1)
        g.set_solution(ur)
    grp = fr.FRGroup(members)
    r = partition.gather(grp.rhs(), ids, u)
    assert rel_l2_rhs(r, whole.rhs()).max() < 1e-12
    with pytest.raises(fr.FRError):
        members[0].set_viscous_scheme(0.5, 0.1)
    grp.close()
    members[0].set_viscous_scheme(0.5, 0.1)
    with pytest.raises(fr.FRError):
        fr.FRGroup(members)
