"""Tiles and schedules of the kernels (Section 3.1: kernel configurations
benchmarked at run time, the fastest kept; independent kernels as parallel
branches of the task graph).  Every schedule runs the same arithmetic per
element, so right-hand sides and RK steps must agree bit for bit; the
autotuner's choice is recorded and applied."""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, ics, mixed_box
from frtest import lib_state

pytestmark = pytest.mark.gpu

BCS = {0: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09), 1: ("extrap",),
       2: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09), 3: ("extrap",)}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _run(spec, p, precision, variant, schedule, physics="ns"):
    g = fr.FRMesh(spec, p, physics=physics, mu=0.02, prandtl=0.71, bcs=BCS,
                  precision=precision)
    g.set_variant(variant)
    g.set_solution(lib_state(g, ics.flow3d))
    g.rk_step("rk45", 1e-4, 1)          # resolves the family
    g.set_solution(lib_state(g, ics.flow3d))
    if schedule:
        g.set_schedule(**schedule)
    r = g.rhs()
    g.rk_step("rk45", 1e-4, 2)
    out = (r, g.get_solution(), g.schedule())
    g.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_hex_tiles_are_bitwise_equal(p, precision):
    spec = box_hex((5, 4, 3), perturb=0.1)
    ref = _run(spec, p, precision, "sumfact", None)
    tmax = ref[2]["hex"]
    assert tmax["grad"] == 0
    for t in (1, 2, 3):
        if t > (1 if (p + 1) ** 3 >= 256 else 256 // (p + 1) ** 3):
            continue
        got = _run(spec, p, precision, "sumfact",
                   {"tiles": {"hex": (t, t)}, "face_block": 128})
        assert got[2]["hex"]["grad"] == t and got[2]["face_block"] == 128
        for a, b in ((got[0], ref[0]), (got[1], ref[1])):
            assert np.array_equal(a["hex"], b["hex"])


@pytest.mark.parametrize("variant", ["sumfact", "tensor"])
def test_mixed_mesh_schedules_are_bitwise_equal(variant):
    spec = mixed_box(n=4, x_pri=0.34, x_tet=0.67, perturb=0.05)
    ref = _run(spec, 3, "fp32", variant, None)
    got = _run(spec, 3, "fp32", variant,
               {"tiles": {"pri": (1, 1), "tet": (1, 1), "hex": (1, 2)},
                "face_block": 512, "parallel_types": True})
    assert got[2]["parallel_types"] and got[2]["face_block"] == 512
    for a, b in ((got[0], ref[0]), (got[1], ref[1])):
        for t in a:
            assert np.array_equal(a[t], b[t])


def test_autotuner_picks_tiles_and_schedule():
    spec = mixed_box(n=8, x_pri=0.34, x_tet=0.67, perturb=0.05)
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71, bcs=BCS,
                  precision="fp32")
    u0 = lib_state(g, ics.flow3d)
    g.set_solution(u0)
    g.rk_step("rk4", 1e-4, 2)
    sc = g.schedule()
    assert sc["ms_default"] > 0 and 0 < sc["ms_tuned"] <= sc["ms_default"] * 1.05
    assert sc["face_block"] in (128, 256, 512)
    for t in ("hex", "pri", "tet"):
        assert sc[t]["grad"] >= 0 and sc[t]["vol"] >= 0
    # the tuned schedule, replayed on a fresh handle, gives the same steps
    h = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71, bcs=BCS,
                  precision="fp32")
    h.set_variant(g.tuning()[0])
    h.set_solution(u0)
    h.rk_step("rk4", 1e-4, 1)
    h.set_solution(u0)
    h.set_schedule(tiles={t: (sc[t]["grad"], sc[t]["vol"]) for t in ("hex", "pri", "tet")},
                   face_block=sc["face_block"], parallel_types=sc["parallel_types"])
    h.rk_step("rk4", 1e-4, 2)
    # a fixed tensor family runs every capable type on the tensor cores; the
    # tuner may have kept some on CUDA cores, which rounds differently
    hs = h.schedule()
    if all(sc[t]["tensor_grad"] == hs[t]["tensor_grad"]
           and sc[t]["tensor_vol"] == hs[t]["tensor_vol"] for t in ("pri", "tet")):
        for t in g.types:
            assert np.array_equal(g.get_solution()[t], h.get_solution()[t])


def test_schedule_rejects_bad_values():
    g = fr.FRMesh(box_hex((2, 2, 2)), 3, physics="euler")
    with pytest.raises(fr.FRError):
        g.set_schedule(face_block=100)
    with pytest.raises(fr.FRError):
        g.set_schedule(tiles={"hex": (99, 1)})
