"""Exchange between processes, host side, with gloo ranks on the CPU
(Section 3.3 partitions; the exchange of Section 3.1, "Multi-node
capabilities").  Every rank builds its part as a host-only handle, the
ranks all-gather their exchange faces, the library matches them
(fr_exchange_setup), and each rank sends the positions of its exchanged
points in message order to every partner: the partner must receive, point
for point, its own points' positions (up to a periodic translation), and
both directions must carry the same counts."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _min_image(d, periodic):
    """Smallest |d + sum k_i T_i| over k_i in {-1, 0, 1}."""
    best = np.linalg.norm(d, axis=-1)
    shifts = [np.zeros(3)]
    for T in periodic:
        shifts = [s + k * np.asarray(T, float) for s in shifts for k in (-1, 0, 1)]
    for s in shifts:
        best = np.minimum(best, np.linalg.norm(d + s, axis=-1))
    return best


def _rank(rank, world, port, case, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from frinputs import box_hex, mixed_box
    import paper_2408_16509_gb300 as fr
    from paper_2408_16509_gb300 import partition
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    spec = {"hex": lambda: box_hex((4, 3, 3), perturb=0.1),
            "mixed": lambda: mixed_box(n=4, x_pri=0.34, x_tet=0.67, perturb=0.05)}[case]()
    bcs = {k: ("extrap",) for k in range(6)}
    subs, ids, _ = partition.split(spec, world, "weighted", halo_last=True)
    g = fr.FRMesh(subs[rank], 2, bcs=partition.exchange_bcs(bcs), device=-1)
    mine = g.exchange_faces()
    allf = [None] * world
    dist.all_gather_object(allf, tuple(np.asarray(a).tolist() for a in mine))
    counts = g.exchange_setup(rank, [tuple(np.asarray(a) for a in x) for x in allf])
    lst = g.exchange_list()
    bx, kind = g.boundary_points()
    assert np.all(kind[lst] == 2)
    n_x = int(np.sum(kind == 2))
    assert len(lst) == n_x == counts.sum() and len(set(lst.tolist())) == n_x
    offs = np.concatenate([[0], np.cumsum(counts)])
    allc = [None] * world
    dist.all_gather_object(allc, counts.tolist())
    worst = 0.0
    for q in range(world):
        assert allc[q][rank] == counts[q]
        if q == rank or counts[q] == 0:
            continue
        mine_x = torch.from_numpy(np.ascontiguousarray(bx[lst[offs[q]:offs[q + 1]]]))
        theirs = torch.empty_like(mine_x)
        reqs = [dist.isend(mine_x, q), dist.irecv(theirs, q)]
        for r in reqs:
            r.wait()
        worst = max(worst, float(_min_image(mine_x.numpy() - theirs.numpy(),
                                            spec.periodic).max()))
    out[rank] = (worst, int(counts.sum()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("hex", 2), ("hex", 3), ("mixed", 2)])
def test_exchange_matching_between_gloo_ranks(case, world):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, case, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(world):
            worst, n = out[r]
            assert n > 0 and worst < 1e-12, (r, worst)
