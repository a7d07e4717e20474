"""The boundary's calls on the GPU, through the C ABI: fr_rhs with host and
device outputs (Section 2 right-hand side), solution upload and download
from device arrays in FP64 and FP32, and fr_stats (counters and device
timings of the timed calls, filter counters of Section 3.2)."""
import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, ics, mixed_box
from frtest import lib_state, oracle_state, rel_l2_rhs
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh

pytestmark = pytest.mark.gpu

BCS = {0: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09), 1: ("extrap",),
       2: ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09), 3: ("extrap",)}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _mixed(physics="ns", precision="fp64"):
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    g = fr.FRMesh(spec, 3, physics=physics, mu=0.02, prandtl=0.71, bcs=BCS,
                  precision=precision)
    g.set_solution(lib_state(g, ics.flow3d))
    return spec, g


def test_rhs_host_and_device_outputs_agree_with_oracle():
    torch = pytest.importorskip("torch")
    spec, g = _mixed()
    r = g.rhs(t=0.25)
    per_type = g.get_rhs()
    n = sum(v.size for v in r.values())
    dev = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    g.rhs_device(t=0.5, out=dev)
    g.sync()
    flat = dev.cpu().numpy()
    off = 0
    for t in g.types:
        assert np.array_equal(r[t], per_type[t])
        assert np.array_equal(flat[off:off + r[t].size].reshape(r[t].shape), r[t])
        off += r[t].size
    o = OracleMesh(spec.as_dict(), 3)
    osys = FRSystem(o, "ns", mu=0.02, pr=0.71, bcs=BCS)
    err = rel_l2_rhs(r, osys.rhs(oracle_state(o, ics.flow3d)))
    assert err.max() < 1e-12, err
    assert g.stats()["t_last"] == 0.5


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_solution_device_arrays_fp64_and_fp32(precision):
    torch = pytest.importorskip("torch")
    _, g = _mixed("euler", precision)
    u = g.get_solution()
    for t in g.types:
        d32 = torch.from_numpy(u[t].astype(np.float32)).cuda()
        g.set_solution_device(t, d32)
        g.sync()
        back = g.get_solution()[t]
        assert np.array_equal(back, u[t].astype(np.float32).astype(np.float64))
        out32 = torch.empty_like(d32)
        g.get_solution_device(t, out32)
        out64 = torch.empty(d32.shape, dtype=torch.float64, device="cuda")
        g.get_solution_device(t, out64)
        g.sync()
        assert torch.equal(out32, d32)
        assert np.array_equal(out64.cpu().numpy(), back)
    with pytest.raises(ValueError):
        g.set_solution_device(g.types[0], torch.zeros(3, dtype=torch.int32, device="cuda"))


def test_stats_counts_stages_and_times_calls():
    spec = box_hex((4, 4, 4), perturb=0.1)
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, prandtl=0.71)
    g.set_solution(lib_state(g, ics.flow3d))
    g.set_variant("sumfact")
    g.stats(reset=True)
    g.rhs(t=1.5)
    g.rhs(t=2.0)
    g.rk_step("rk45", 1e-4, 3)
    g.rk_step("rk4", 1e-4, 2)
    prof = g.profile_step("rk45", 1e-4)
    ok, err, dt = g.rk_adaptive_step(1e-4, fr.AdaptCtl(1e-6, 1e-6, 1.0, 0))
    st = g.stats()
    assert st["rhs_calls"] == 2 and st["rk_steps"] == 3 + 2 + 1
    assert st["rk_attempts"] == 1 and st["rk_rejected"] == (0 if ok else 1)
    assert st["stages"] == 2 + 3 * 5 + 2 * 4 + 5 + 5
    assert st["ms_device"] > 0
    assert st["t_last"] == 2.0 and st["kernel_family"] == "sumfact"
    assert st["launches"]["volume"] == prof["volume"][1] == 5
    assert st["kernel_ms"]["volume"] == pytest.approx(prof["volume"][0])
    st2 = g.stats(reset=True)
    assert st2["ms_device"] >= st["ms_device"]
    st3 = g.stats()
    assert st3["rhs_calls"] == 0 and st3["stages"] == 0 and st3["ms_device"] == 0


def test_stats_filter_counters_match_filter_stats():
    spec = box_hex((64, 2, 2), lo=(-5.0, 0, 0), hi=(5.0, 0.3125, 0.3125),
                   periodic=(1, 2))
    post = ics.SHU_OSHER_POST
    bcs = {0: ("state", post[0], post[1], 0.0, 0.0, post[2]), 1: ("extrap",)}
    g = fr.FRMesh(spec, 3, physics="euler", bcs=bcs, precision="fp32")
    g.set_solution(lib_state(g, ics.shu_osher))
    g.filter_enable(True)
    g.filter_stats(reset=True)
    g.stats(reset=True)
    g.rk_step("rk4", 2e-3, 3)
    st = g.stats()
    fs = g.filter_stats()
    assert st["filtered"] == fs["filtered"] > 0
    assert st["filter_evals"] == fs["evals"]
    assert st["predictor_used"] == fs["guessed"] == 0
