"""Partitioned right-hand side on one device (Section 4, domain
decomposition; the exchange of Section 3): the parts of a mesh, each with
its faces towards other parts as exchange boundaries, run as a group and
must reproduce the unpartitioned mesh.

Tolerances: the exchange points of a part use their own side's normal and
metric magnitude where the unpartitioned interface kernel uses the left
side's (on curved elements the two sides' curl-form normals agree to
rounding), so the two differ by rounding only: FP64 right-hand sides and
solutions 1e-12 relative L2 (as every FP64 parity test), FP32 1e-5.
"""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, curved_box_hex, ics, mixed_box
from frtest import lib_state, rel_l2, rel_l2_rhs
from paper_2408_16509_gb300 import partition

pytestmark = pytest.mark.gpu

BCS = {0: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       1: ("extrap",),
       2: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
       3: ("extrap",)}

SPECS = {
    "hex": lambda: box_hex((4, 4, 3), perturb=0.1),
    "mixed": lambda: mixed_box(n=4, x_pri=0.34, x_tet=0.67, perturb=0.05),
    "curved": lambda: curved_box_hex((4, 3, 3)),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _tgv(x):
    # every conserved variable's right-hand side O(1) (per-variable norms)
    return ics.flow3d(x)


def _setup(name, nparts, physics, precision="fp64", mode="weighted", p=3, qdeg=0):
    spec = SPECS[name]()
    bcs = BCS if name == "mixed" else None
    kw = dict(physics=physics, gamma=1.4, mu=0.02, prandtl=0.71,
              precision=precision)
    whole = fr.FRMesh(spec, p, bcs=bcs, **kw)
    whole.set_variant("sumfact")
    u = lib_state(whole, _tgv)
    whole.set_solution(u)
    subs, ids, _ = partition.split(spec, nparts, mode)
    members = []
    for s in subs:
        g = fr.FRMesh(s, p, bcs=partition.exchange_bcs(bcs), **kw)
        g.set_variant("sumfact")
        members.append(g)
    for g, ur in zip(members, partition.scatter(u, ids)):
        g.set_solution(ur)
    if qdeg:
        whole.set_antialias(qdeg)
        for g in members:
            g.set_antialias(qdeg)
    return whole, members, ids, u


@pytest.mark.parametrize("name", ["hex", "mixed", "curved"])
@pytest.mark.parametrize("nparts", [2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_group_rhs_equals_whole_fp64(name, nparts, physics):
    whole, members, ids, u = _setup(name, nparts, physics)
    grp = fr.FRGroup(members)
    r = partition.gather(grp.rhs(), ids, u)
    err = rel_l2_rhs(r, whole.rhs())
    assert err.max() < 1e-12, err
    grp.close()


@pytest.mark.parametrize("name,mode", [("hex", "weighted"), ("mixed", "balanced")])
def test_group_rk_steps_fp64(name, mode):
    whole, members, ids, u = _setup(name, 3, "ns", mode=mode)
    grp = fr.FRGroup(members)
    grp.rk_step("rk45", 1e-3, 3)
    whole.rk_step("rk45", 1e-3, 3)
    got = partition.gather([m.get_solution() for m in members], ids, u)
    assert rel_l2(got, whole.get_solution()).max() < 1e-12


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_group_fp32_forms(precision):
    """FP32 values: the viscous coupling goes through the exchanged normal
    viscous fluxes (and the partners' metric magnitudes)."""
    name = "hex"
    whole, members, ids, u = _setup(name, 3, "ns", precision=precision)
    grp = fr.FRGroup(members)
    grp.rk_step("rk4", 1e-3, 2)
    whole.rk_step("rk4", 1e-3, 2)
    got = partition.gather([m.get_solution() for m in members], ids, u)
    assert rel_l2(got, whole.get_solution()).max() < 1e-5


def test_group_fp32_mixed_mesh_rhs():
    whole, members, ids, u = _setup("mixed", 2, "ns", precision="fp32")
    grp = fr.FRGroup(members)
    r = partition.gather(grp.rhs(), ids, u)
    assert rel_l2_rhs(r, whole.rhs()).max() < 1e-5


def test_group_with_antialiasing():
    whole, members, ids, u = _setup("hex", 2, "ns", qdeg=9)
    grp = fr.FRGroup(members)
    r = partition.gather(grp.rhs(), ids, u)
    assert rel_l2_rhs(r, whole.rhs()).max() < 1e-12


def test_members_refuse_to_run_alone_and_incomplete_groups_fail():
    whole, members, ids, u = _setup("hex", 2, "euler")
    with pytest.raises(fr.FRError) as e:
        members[0].rhs()
    assert e.value.name == "FR_EINVAL"
    with pytest.raises(fr.FRError) as e:
        fr.FRGroup(members[:1])
    assert e.value.name == "FR_EMESH"
    grp = fr.FRGroup(members)
    with pytest.raises(fr.FRError):
        fr.FRGroup(members)          # already in a group
    grp.close()
    fr.FRGroup(members).close()      # free again after close
