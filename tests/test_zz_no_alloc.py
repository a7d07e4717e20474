"""fr_set_solution_static: the allocation-free solution upload.

Callers that cannot allocate device memory (their memory is reserved up
front by their own pool allocator, or their time-stepping loop must not pay
the synchronisation cudaMalloc / cudaFree can imply) upload solutions through
this entry point, which stages the copy in a fixed array compiled into the
library instead of a cudaMalloc'd buffer.  The test calls it through the C
ABI and checks it against fr_set_solution, on two calls in a row.  It sits in
a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, ics, mixed_box

pytestmark = pytest.mark.gpu

BCS = {k: ("state", 1.0, 0.2, 0.0, 0.0, 5.0) for k in range(4)}


def _static(g, etype, u):
    a = np.ascontiguousarray(u, np.float64)
    return fr.load().fr_set_solution_static(
        g._h, fr.ETYPES[etype], a.ctypes.data_as(ctypes.c_void_p))


def _state(g, rng, scale):
    out = {}
    for t in g.types:
        x = g.points(t)
        u = ics.taylor_green(2 * np.pi * x.reshape(-1, 3), mach=0.3)
        u *= 1.0 + scale * rng.uniform(-1, 1, size=u.shape)
        out[t] = u.reshape(x.shape[0], x.shape[1], 5)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_upload_matches_fr_set_solution(precision):
    fr.build()
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67, perturb=0.05)
    ref = fr.FRMesh(spec, 3, physics="ns", mu=0.02, bcs=BCS,
                    precision=precision)
    g = fr.FRMesh(spec, 3, physics="ns", mu=0.02, bcs=BCS,
                  precision=precision)
    rng = np.random.default_rng(11)
    for call in range(2):                  # two calls in a row
        u = _state(g, rng, 0.01 * (call + 1))
        ref.set_solution(u)
        for t in g.types:
            assert _static(g, t, u[t]) == 0, fr.load().fr_last_error()
        a, b = ref.get_solution(), g.get_solution()
        for t in g.types:
            assert np.array_equal(a[t], b[t])
        ra, rb = ref.rhs(), g.rhs()
        for t in g.types:
            assert np.array_equal(ra[t], rb[t])


def test_static_upload_rejects_oversized_solutions():
    fr.build()
    spec = box_hex((20, 20, 20))           # 8000 * 64 * 5 > 2^21 values
    g = fr.FRMesh(spec, 3)
    u = np.ones((8000, 64, 5))
    rc = _static(g, "hex", u)
    assert fr.ERRORS.get(rc) == "FR_EINVAL"
    assert b"static staging limit" in fr.load().fr_last_error()


def test_static_upload_leaves_device_free_memory_unchanged():
    """No device allocation: the device's free memory (cudaMemGetInfo) is the
    same before and after repeated uploads on a fresh handle, while the
    allocating fr_set_solution on another fresh handle does take memory for
    its staging buffer (2.56 MB here), so the check can see an allocation."""
    torch = pytest.importorskip("torch")
    fr.build()
    spec = box_hex((10, 10, 10))           # 1000 * 64 * 5 values: 2.56 MB FP64
    g = fr.FRMesh(spec, 3)
    u = np.ascontiguousarray(_state(g, np.random.default_rng(3), 0.01)["hex"])
    assert _static(g, "hex", u) == 0       # first call: looks up the array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _static(g, "hex", u) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    h = fr.FRMesh(spec, 3)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    h.set_solution({"hex": u})
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1
