"""A partitioned mesh with one part per process (Section 3.3), the exchange
(Section 3.1, "Multi-node capabilities") carried by torch.distributed over
gloo through pinned host buffers.  The two processes share this run's one
GPU; their kernels never wait on each other (the host transports between
phases).  The parts' RK steps must reproduce the whole mesh's (FP64 1e-12,
FP32 1e-6: each side rounds with its own unit normal) and the oracle's
(FP64 1e-12), with and without the overlap of transport and interior work
(which must agree bit for bit)."""
import os
import socket
import sys

import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, ics, mixed_box
from frtest import lib_state, oracle_state, rel_l2
from oracle import rk
from oracle.fr import FRSystem
from oracle.mesh import FRMesh as OracleMesh

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAR = ("state", 1.0, 0.4, 0.1, 0.0, 1.0 / 1.4 / 0.09)
BCS = {0: FAR, 1: ("extrap",), 2: FAR, 3: ("extrap",)}


def _spec(case):
    if case == "hex":
        return box_hex((5, 4, 3), perturb=0.1)
    return mixed_box(n=4, x_pri=0.34, x_tet=0.67, perturb=0.05)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, case, physics, prec, overlap, steps, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_2408_16509_gb300 as frr
    from frinputs import ics as ics_
    from frtest import lib_state as ls
    from paper_2408_16509_gb300 import partition
    from paper_2408_16509_gb300.distributed import DistributedPart
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    subs, ids, _ = partition.split(_spec(case), world, "weighted", halo_last=True)
    g = frr.FRMesh(subs[rank], 2, physics=physics, mu=0.02, prandtl=0.71,
                   bcs=partition.exchange_bcs(BCS), precision=prec)
    g.set_variant("sumfact")
    g.set_solution(ls(g, ics_.flow3d))
    part = DistributedPart(g, dist, torch, overlap=overlap)
    part.rk_step("rk45", 2e-4, steps)
    st = g.stats()
    out[rank] = ({t: a for t, a in g.get_solution().items()}, ids[rank],
                 int(part.counts.sum()), st["rk_steps"])
    dist.barrier()
    dist.destroy_process_group()


def _run_ranks(world, case, physics, prec, overlap, steps):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, case, physics, prec,
                                                 overlap, steps, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(600)
        assert all(p.exitcode == 0 for p in procs)
        return [out[r] for r in range(world)]


def _gathered(res, like):
    from paper_2408_16509_gb300 import partition
    return partition.gather([r[0] for r in res], [r[1] for r in res], like)


@pytest.mark.parametrize("case,physics,world", [("hex", "ns", 2), ("mixed", "ns", 2),
                                                ("hex", "euler", 3)])
def test_parts_in_processes_equal_whole_mesh_and_oracle(case, physics, world):
    steps = 3
    spec = _spec(case)
    whole = fr.FRMesh(spec, 2, physics=physics, mu=0.02, prandtl=0.71, bcs=BCS)
    whole.set_variant("sumfact")
    whole.set_solution(lib_state(whole, ics.flow3d))
    whole.rk_step("rk45", 2e-4, steps)
    ref = whole.get_solution()
    res = _run_ranks(world, case, physics, "fp64", True, steps)
    assert all(r[2] > 0 and r[3] == steps for r in res)
    got = _gathered(res, ref)
    assert rel_l2(got, ref).max() < 1e-12
    o = OracleMesh(spec.as_dict(), 2)
    osys = FRSystem(o, physics, mu=0.02, pr=0.71, bcs=BCS)
    u = oracle_state(o, ics.flow3d)
    for _ in range(steps):
        u = rk.step(osys.rhs, u, 2e-4, "rk45")
    assert rel_l2(got, u).max() < 1e-12
    plain = _gathered(_run_ranks(world, case, physics, "fp64", False, steps), ref)
    for t in got:
        assert np.array_equal(got[t], plain[t])


def test_parts_in_processes_fp32():
    spec = _spec("hex")
    whole = fr.FRMesh(spec, 2, physics="ns", mu=0.02, prandtl=0.71, bcs=BCS,
                      precision="fp32")
    whole.set_variant("sumfact")
    whole.set_solution(lib_state(whole, ics.flow3d))
    whole.rk_step("rk45", 2e-4, 3)
    ref = whole.get_solution()
    got = _gathered(_run_ranks(2, "hex", "ns", "fp32", True, 3), ref)
    assert rel_l2(got, ref).max() < 1e-6
