"""GPU parity on curved hexahedra, prisms and tetrahedra ("Curved Elements",
Section 3.4): the
library's quadratic-map geometry (conservative curl-form metric, exact
det J) and every kernel family that can run on it, against the oracle.

Tolerances are those of the straight-element tests: FP64 right-hand sides
1e-12 relative L2 (5e-12 at p = 4), FP64 solutions 1e-12, FP32 solutions
1e-6.  Free-stream preservation is a property at any size: a uniform state
gives a right-hand side at round-off, bounded by the oracle's own FP64
residual on the same mesh (times the unit round-off ratio for FP32).
"""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import curved_box_hex, ics
from frtest import lib_state, oracle_state, rel_l2, rel_l2_rhs
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh

pytestmark = pytest.mark.gpu

ZBCS = {4: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09),
        5: ("extrap",)}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _tgv(x):
    # every conserved variable's right-hand side O(1): a per-variable
    # relative norm then measures each one against a comparable scale
    return ics.flow3d(x)


def _pair(spec, p, physics, bcs=None, precision="fp64"):
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, physics, gamma=1.4, mu=0.02, pr=0.71, bcs=bcs)
    g = fr.FRMesh(spec, p, physics=physics, gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=bcs, precision=precision)
    assert np.abs(g.points("hex") - o.upts_x["hex"]).max() < 1e-14
    return o, osys, g


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_curved_rhs_fp64(p, physics):
    # 3x3x2 = 18 curved elements: several CTAs and a ragged last one
    spec = curved_box_hex((3, 3, 2))
    o, osys, g = _pair(spec, p, physics)
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < (5e-12 if p == 4 else 1e-12), err


@pytest.mark.parametrize("variant", ["dense", "sumfact"])
def test_curved_boundaries_and_rk_fp64(variant):
    """Curved elements on the z boundaries (inflow state and extrapolation),
    three RK4(3)5[2R+] steps, both FP64 hexahedron families."""
    spec = curved_box_hex((3, 2, 3), periodic=(0, 1))
    o, osys, g = _pair(spec, 3, "ns", bcs=ZBCS)
    g.set_variant(variant)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    err = rel_l2_rhs(g.rhs(), osys.rhs(u))
    assert err.max() < 1e-12, err
    for _ in range(3):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 3)
    assert rel_l2(g.get_solution(), u).max() < 1e-12


@pytest.mark.parametrize("variant", ["sumfact", "sumfact_vertex", "dense"])
def test_curved_fp32_families(variant):
    """FP32 values on curved elements.  The vertex-metric family rebuilds
    trilinear metrics in the kernel, so a request for it on a curved mesh
    runs the table-metric sum-factorised family instead."""
    spec = curved_box_hex((3, 3, 2))
    o, osys, g = _pair(spec, 3, "ns", precision="fp32")
    g.set_variant(variant)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    assert rel_l2(g.get_solution(), u).max() < 1e-6
    active, _ = g.tuning()
    assert active != "sumfact_vertex"


def test_curved_autotuner_excludes_vertex_metrics():
    spec = curved_box_hex((5, 5, 5))
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71, precision="fp32")
    g.set_solution(lib_state(g, _tgv))
    g.rk_step("rk45", 1e-3, 1)
    active, ms = g.tuning()
    assert "sumfact_vertex" not in ms and active in ms


@pytest.fixture(scope="module")
def oracle_free_stream_16():
    """The oracle's FP64 free-stream residual on 16^3 curved hexahedra, p=3:
    round-off only (its metric is discretely divergence-free), and it grows
    with the cells per unit length (about n^3 on the unit box)."""
    o = OracleMesh(curved_box_hex((16, 16, 16)).as_dict(), 3)
    osys = FRSystem(o, "ns", gamma=1.4, mu=0.02, pr=0.71)
    return np.abs(osys.rhs(oracle_state(o, ics.uniform))["hex"]).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_curved_free_stream_at_size(precision, oracle_free_stream_16):
    """16^3 curved hexahedra, p = 3: a uniform state stays uniform to
    round-off.  Bound: 4x the oracle's FP64 residual on the same mesh, scaled
    by the unit round-off ratio for FP32 values."""
    spec = curved_box_hex((16, 16, 16))
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71,
                  precision=precision)
    g.set_solution(lib_state(g, ics.uniform))
    r = np.abs(g.rhs()["hex"]).max()
    ratio = 1.0 if precision == "fp64" else 2.0 ** -24 / 2.0 ** -53
    assert 0 < oracle_free_stream_16 < 1e-9
    assert r <= 4 * ratio * oracle_free_stream_16, (r, oracle_free_stream_16)


# ---------------------------------------------------------------- simplices
MIXED_BCS = {0: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09), 1: ("extrap",),
             2: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09), 3: ("extrap",)}


def _curved_mixed(n=3, **kw):
    from frinputs import curved_mixed_box
    return curved_mixed_box(n=n, **kw)


def _pair_mixed(spec, p, physics, precision="fp64", bcs=MIXED_BCS):
    o = OracleMesh(spec.as_dict(), p)
    osys = FRSystem(o, physics, gamma=1.4, mu=0.02, pr=0.71, bcs=bcs)
    g = fr.FRMesh(spec, p, physics=physics, gamma=1.4, mu=0.02, prandtl=0.71,
                  bcs=bcs, precision=precision)
    for t in g.types:
        assert np.abs(g.points(t) - o.upts_x[t]).max() < 1e-14
    return o, osys, g


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_curved_mixed_rhs_fp64(p, physics):
    """Curved hexahedra, prisms (18-node maps) and tetrahedra (10-node maps)
    against the oracle, FP64, 1e-12 per conserved variable."""
    o, osys, g = _pair_mixed(_curved_mixed(), p, physics)
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < (5e-12 if p == 4 else 1e-12), err


def test_curved_prisms_and_tets_rhs_fp64():
    spec = _curved_mixed(x_pri=0.0, x_tet=0.5, periodic_x=False)
    o, osys, g = _pair_mixed(spec, 3, "ns")
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < 1e-12, err


@pytest.mark.parametrize("precision,variant,tol", [("fp64", "sumfact", 1e-12),
                                                   ("fp32", "sumfact", 1e-6),
                                                   ("fp32", "tensor", 1e-6)])
def test_curved_mixed_rk_steps(precision, variant, tol):
    o, osys, g = _pair_mixed(_curved_mixed(), 3, "ns", precision=precision)
    g.set_variant(variant)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 2e-4, "rk45")
    g.rk_step("rk45", 2e-4, 2)
    err = rel_l2(g.get_solution(), u)
    assert err.max() < tol, err


@pytest.mark.parametrize("p", [2, 3])
def test_curved_mixed_free_stream_at_size(p):
    """A uniform state on 16^3 cells of curved hexahedra, prisms and
    tetrahedra: the right-hand side is round-off of the flux divergence,
    whose scale is |F| (p+1)^2 / h (|F| ~ 4 for this state): bounded by
    1e-11 of that.  (The pointwise metric leaves O(1) at p = 2.)"""
    n = 16
    spec = _curved_mixed(n=n)
    far = ("state", 1.0, 0.5, 0.3, 0.2, 1.0)
    g = fr.FRMesh(spec, p, physics="ns", mu=1e-3, prandtl=0.71,
                  bcs={k: far for k in range(4)})
    g.set_solution(lib_state(g, lambda x: ics.uniform(x, vel=(0.5, 0.3, 0.2))))
    r = g.rhs()
    scale = 4.0 * (p + 1) ** 2 * n
    assert max(np.abs(v).max() for v in r.values()) < 1e-11 * scale


# ---------------------------------------------------------------- cubic maps
@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_cubic_hex_rhs_fp64(p, physics):
    """64-node (cubic) hexahedron maps, FP64, against the oracle."""
    spec = curved_box_hex((3, 3, 2), order=3)
    o, osys, g = _pair(spec, p, physics)
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < (5e-12 if p == 4 else 1e-12), err


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_cubic_hex_rk_steps(precision, tol):
    spec = curved_box_hex((3, 3, 2), order=3)
    o, osys, g = _pair(spec, 3, "ns", precision=precision)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 1e-3, "rk45")
    g.rk_step("rk45", 1e-3, 2)
    err = rel_l2(g.get_solution(), u)
    assert err.max() < tol, err


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("physics", ["euler", "ns"])
def test_cubic_mixed_rhs_fp64(p, physics):
    """Cubic maps on every type (64-node hexahedra, 40-node prisms, 20-node
    tetrahedra) against the oracle, FP64, per conserved variable, 5e-12.
    The bound is set by the geometry both sides start from: the library's
    host metrics of cubic simplices equal the oracle's to 5e-13 of their
    scale (different summation orders in a curl form that cancels products
    X_l dX_m some ten times larger than S), and on this mesh the oracle's
    own right-hand side moves by 1e-12 to 1e-11 per variable when its
    metrics are perturbed at random by 2e-13 relative (p = 2, 3).  At
    p = 3 the GPU lands 2e-12 from the oracle."""
    o, osys, g = _pair_mixed(_curved_mixed(order=3), p, physics)
    g.set_solution(lib_state(g, _tgv))
    err = rel_l2_rhs(g.rhs(), osys.rhs(oracle_state(o, _tgv)))
    assert err.max() < 5e-12, err


@pytest.mark.parametrize("precision,variant,tol", [("fp64", "sumfact", 1e-12),
                                                   ("fp32", "sumfact", 1e-6),
                                                   ("fp32", "tensor", 1e-6)])
def test_cubic_mixed_rk_steps(precision, variant, tol):
    o, osys, g = _pair_mixed(_curved_mixed(order=3), 3, "ns", precision=precision)
    g.set_variant(variant)
    g.set_solution(lib_state(g, _tgv))
    u = oracle_state(o, _tgv)
    for _ in range(2):
        u = rk.step(osys.rhs, u, 2e-4, "rk45")
    g.rk_step("rk45", 2e-4, 2)
    err = rel_l2(g.get_solution(), u)
    assert err.max() < tol, err
