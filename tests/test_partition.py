"""Domain decomposition on the host (Section 4, "Mixed Elements and Domain
Decomposition"): element adjacency, weighted and balanced partitioning,
the faces between parts, and sub-meshes that build with those faces as
exchange boundaries.  No GPU: host-only handles.  The per-rank set-up of a
partitioned run is also checked with two gloo ranks."""
import os
import socket
import sys

import numpy as np
import pytest

import paper_2408_16509_gb300 as fr
from frinputs import box_hex, curved_box_hex, mixed_box
from paper_2408_16509_gb300 import partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIXED_BCS = {k: ("extrap",) for k in range(6)}


@pytest.fixture(scope="module", autouse=True)
def built():
    fr.build()


def _host(spec, bcs=None):
    return fr.FRMesh(spec, 1, bcs=bcs or MIXED_BCS, device=-1)


def _global_adjacency(m):
    return {t: m.adjacency(t) for t in m.types}


@pytest.mark.parametrize("name", ["hex_periodic", "mixed"])
def test_adjacency_is_symmetric(name):
    spec = {"hex_periodic": lambda: box_hex((3, 2, 2), perturb=0.1),
            "mixed": lambda: mixed_box(n=3, x_pri=0.34, x_tet=0.67)}[name]()
    m = _host(spec)
    adj = _global_adjacency(m)
    offs = np.cumsum([0] + [m.info(t)[0] for t in m.types])
    nbr = np.concatenate([adj[t].ravel() for t in m.types])
    owner = np.concatenate([np.repeat(np.arange(offs[i], offs[i + 1]), adj[t].shape[1])
                            for i, t in enumerate(m.types)])
    inner = nbr >= 0
    pairs = set(zip(owner[inner].tolist(), nbr[inner].tolist()))
    assert all((b, a) in pairs for a, b in pairs)
    if name == "hex_periodic":
        assert inner.all()          # fully periodic box: no boundary
    else:
        n_bnd = int((~inner).sum())
        assert n_bnd == len(spec.bfaces)


@pytest.mark.parametrize("nparts", [2, 3, 4, 7])
def test_weighted_partition_balances_weight(nparts):
    spec = mixed_box(n=6, x_pri=0.34, x_tet=0.67)
    m = _host(spec)
    w = np.array([1.0, 0.6, 0.35])
    part = m.partition(nparts, "weighted", w)
    kinds = np.concatenate([np.full(m.info(t)[0], i) for i, t in
                            enumerate(m.types)])
    wt = w[kinds]
    load = np.bincount(part, weights=wt, minlength=nparts)
    assert part.min() == 0 and part.max() == nparts - 1
    assert load.max() - wt.sum() / nparts <= 3 * wt.max()


@pytest.mark.parametrize("nparts", [2, 4])
def test_balanced_partition_equal_counts_per_type(nparts):
    spec = mixed_box(n=6, x_pri=0.34, x_tet=0.67)
    m = _host(spec)
    part = m.partition(nparts, "balanced")
    off = 0
    for t in m.types:
        ne = m.info(t)[0]
        cnt = np.bincount(part[off:off + ne], minlength=nparts)
        assert cnt.max() - cnt.min() <= 2, (t, cnt)
        off += ne


def test_partition_rejects_bad_arguments():
    m = _host(box_hex((2, 2, 2)))
    with pytest.raises(fr.FRError):
        m.partition(0)
    with pytest.raises(fr.FRError):
        m.partition(2, "weighted", [1.0, -1.0, 1.0])


@pytest.mark.parametrize("nparts", [2, 3])
def test_faces_between_parts_match_up(nparts):
    """Part r lists exactly its element faces whose neighbour (periodic
    partners included) lies in another part, and the part-to-part face
    counts are symmetric."""
    spec = mixed_box(n=4, x_pri=0.34, x_tet=0.67)
    m = _host(spec)
    part = m.partition(nparts, "weighted")
    offs = np.cumsum([0] + [m.info(t)[0] for t in m.types])
    C = np.zeros((nparts, nparts), np.int64)
    for i, t in enumerate(m.types):
        adj = m.adjacency(t)
        own = part[offs[i]:offs[i + 1]]
        for f in range(adj.shape[1]):
            nb = adj[:, f]
            sel = nb >= 0
            np.add.at(C, (own[sel], part[nb[sel]]), 1)
    assert np.array_equal(C, C.T)
    for r in range(nparts):
        faces = m.partition_faces(part, r)
        assert len(faces) == C[r].sum() - C[r, r] > 0


@pytest.mark.parametrize("name,nparts,mode", [("hex_periodic", 2, "weighted"),
                                              ("hex_periodic", 4, "weighted"),
                                              ("mixed", 3, "balanced"),
                                              ("curved", 3, "weighted")])
def test_sub_meshes_build_with_exchange_faces(name, nparts, mode):
    spec = {"hex_periodic": lambda: box_hex((4, 4, 2), perturb=0.1),
            "mixed": lambda: mixed_box(n=4, x_pri=0.34, x_tet=0.67, perturb=0.05),
            "curved": lambda: curved_box_hex((4, 3, 2))}[name]()
    subs, ids, part = partition.split(spec, nparts, mode)
    bcs = partition.exchange_bcs(MIXED_BCS)
    total = 0
    for r, s in enumerate(subs):
        g = fr.FRMesh(s, 2, bcs=bcs, device=-1)
        total += g.n_elements()
        npair, nb = g.pair_counts()
        assert nb > 0
    assert total == sum(len(c) for c in spec.elements.values())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_2408_16509_gb300 as frl
    from frinputs import box_hex as bh
    from paper_2408_16509_gb300 import partition as pt
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    spec = bh((4, 4, 4), perturb=0.1)
    subs, ids, part = pt.split(spec, world, "weighted")
    # every rank derives the same partition independently
    h = torch.tensor([int(np.sum(part.astype(np.int64) * np.arange(len(part))))])
    hs = [torch.zeros_like(h) for _ in range(world)]
    dist.all_gather(hs, h)
    same = all(int(x) == int(h) for x in hs)
    # the own part builds with its exchange faces; its count of exchange
    # flux points equals what the other rank sends back (a periodic box
    # split in two shares faces on both sides)
    g = frl.FRMesh(subs[rank], 2, bcs=pt.exchange_bcs({}), device=-1)
    _, nb = g.pair_counts()
    n = torch.tensor([nb])
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n)
    out[rank] = (same, [int(x) for x in ns], len(ids[rank]["hex"]))
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_setup_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(2):
            same, counts, ne = out[r]
            assert same
            assert counts[0] == counts[1] > 0
        assert out[0][2] + out[1][2] == 64


def test_boundary_points_of_a_part():
    """A part of a fully periodic box has only exchange boundary points, at
    the positions of its faces towards the other part."""
    spec = box_hex((4, 2, 2), perturb=0.1)
    subs, ids, part = partition.split(spec, 2, "weighted")
    g = fr.FRMesh(subs[0], 2, bcs=partition.exchange_bcs({}), device=-1)
    x, kind = g.boundary_points()
    _, nb = g.pair_counts()
    assert len(x) == nb > 0 and np.all(kind == 2)
    assert np.all((x >= -1e-12) & (x <= 1 + 1e-12))


def test_groups_refuse_host_only_members():
    """Grouping needs device handles; host-only parts are refused before any
    device call."""
    spec = box_hex((4, 2, 2), perturb=0.1)
    subs, _, _ = partition.split(spec, 2, "weighted")
    parts = [fr.FRMesh(s, 2, bcs=partition.exchange_bcs({}), device=-1) for s in subs]
    with pytest.raises(fr.FRError) as e:
        fr.FRGroup(parts)
    assert e.value.name == "FR_EINVAL"


def test_one_part_has_no_exchange_faces():
    spec = mixed_box(n=3, x_pri=0.34, x_tet=0.67)
    subs, ids, part = partition.split(spec, 1)
    assert np.all(part == 0) and len(subs) == 1
    g = fr.FRMesh(subs[0], 2, bcs=partition.exchange_bcs(MIXED_BCS), device=-1)
    _, kind = g.boundary_points()
    assert not np.any(kind == 2)
