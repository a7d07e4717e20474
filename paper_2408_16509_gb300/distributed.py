"""One part of a partitioned mesh per process (Section 3.3, "Mixed Elements
and Domain Decomposition"), its exchange with the other parts carried by
torch.distributed (Section 3.1, "Multi-node capabilities": the packed face
buffers of the partitions exchanged at every stage).

The library does the work: it matches the exchange points of all ranks
(fr_exchange_setup), packs the traces a partner needs into one device
buffer, unpacks the received ones and runs every stage in phases
(fr_rk_stage).  This module only moves the buffers: device tensors with
NCCL (send/recv on the part's stream), pinned host copies with gloo.  With
``overlap`` the transport of a phase's input runs while the GPU does the
work that needs no exchanged value (fr_rk_stage part 1: interior pairs,
ordinary boundary points and the elements that own no exchange point;
``partition.split(..., halo_last=True)`` puts those first).
"""
import numpy as np

from ._binding import FRMesh  # noqa: F401  (type of `mesh`)

_NV_GRAD = {"fp64": 15, "fp32": 5, "mixed": 5}


class DistributedPart:
    """mesh: this rank's part (an FRMesh built from ``partition.split`` with
    ``partition.exchange_bcs``); dist: torch.distributed, initialised."""

    def __init__(self, mesh, dist, torch, overlap=True, group=None):
        self.mesh, self.dist, self.torch = mesh, dist, torch
        self.group = group
        self.overlap = overlap
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.nccl = dist.get_backend(group) == "nccl"
        mine = mesh.exchange_faces()
        allf = [None] * self.world
        dist.all_gather_object(allf, tuple(np.asarray(a).tolist() for a in mine),
                               group=group)
        per_rank = [tuple(np.asarray(a) for a in x) for x in allf]
        self.counts = mesh.exchange_setup(self.rank, per_rank)
        self.offs = np.concatenate([[0], np.cumsum(self.counts)])
        n = int(self.offs[-1])
        self.dtype = torch.float64 if mesh.precision == "fp64" else torch.float32
        self.stream = torch.cuda.Stream()
        mesh.set_stream(self.stream)
        self.nv = {0: 5, 1: _NV_GRAD[mesh.precision]}
        self.dev = {}
        self.host = {}
        for w, nv in self.nv.items():
            self.dev[w] = (torch.zeros((max(n, 1), nv), dtype=self.dtype, device="cuda"),
                           torch.zeros((max(n, 1), nv), dtype=self.dtype, device="cuda"))
            if not self.nccl:
                self.host[w] = (torch.zeros((max(n, 1), nv), dtype=self.dtype).pin_memory(),
                                torch.zeros((max(n, 1), nv), dtype=self.dtype).pin_memory())
        self.partners = [q for q in range(self.world) if q != self.rank and self.counts[q]]

    def _exchange(self, what, work=None):
        """Pack, send to / receive from every partner, unpack; `work` (the
        launches that need no exchanged value) is issued before waiting."""
        m, t, dist = self.mesh, self.torch, self.dist
        send, recv = self.dev[what]
        m.exchange_pack(what, send)
        if not self.partners:
            if work:
                work()
            return
        if self.nccl:
            with t.cuda.stream(self.stream):
                ops = []
                for q in self.partners:
                    a, b = int(self.offs[q]), int(self.offs[q + 1])
                    ops.append(dist.P2POp(dist.isend, send[a:b], q, self.group, what))
                    ops.append(dist.P2POp(dist.irecv, recv[a:b], q, self.group, what))
                reqs = dist.batch_isend_irecv(ops)
                if work:
                    work()
                for r in reqs:
                    r.wait()
        else:
            hs, hr = self.host[what]
            m.sync()
            hs.copy_(send)
            reqs = []
            for q in self.partners:
                a, b = int(self.offs[q]), int(self.offs[q + 1])
                reqs.append(dist.isend(hs[a:b], q, group=self.group, tag=what))
                reqs.append(dist.irecv(hr[a:b], q, group=self.group, tag=what))
            if work:
                work()           # the GPU runs it while the host transports
            for r in reqs:
                r.wait()
            with t.cuda.stream(self.stream):
                recv.copy_(hr, non_blocking=True)
        m.exchange_unpack(what, recv)

    def rk_step(self, scheme, dt, nsteps=1):
        """nsteps RK steps of the whole partitioned mesh, this rank's part."""
        m = self.mesh
        ns = m.physics == "ns"
        nst = 4 if scheme == "rk4" else 5
        for _ in range(nsteps):
            for st in range(nst):
                if ns:
                    self._phase(scheme, dt, st, 1, 0)
                    self._phase(scheme, dt, st, 2, 1)
                else:
                    self._phase(scheme, dt, st, 2, 0)
        m.sync()

    def _phase(self, scheme, dt, st, phase, what):
        m = self.mesh
        if phase == 2 and m.physics != "ns" and st == 0:
            # Euler: phase 1 is empty, but it starts the step (dt, flags)
            m.rk_stage(scheme, dt, 0, 1, 1 if self.overlap else 0)
        if self.overlap:
            self._exchange(what, lambda: m.rk_stage(scheme, dt, st, phase, 1))
            m.rk_stage(scheme, dt, st, phase, 2)
        else:
            self._exchange(what)
            m.rk_stage(scheme, dt, st, phase, 0)
