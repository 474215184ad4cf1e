"""Domain decomposition of one ADER-DG problem along the depth-first (space-
filling-curve) cell order (paper Sec. 3, distributed memory).

Each rank holds a partitioned context (``ader_partition``): its owned cells
plus ghost cells, whose face data (Q-bar, F-bar) arrive once per step from
their owners.  A step on every rank is

    predict skeleton cells (partition-boundary and transition cells)
    pack the face data each neighbour needs         -> exchange starts
    predict enclave cells                           (overlaps the exchange)
    unpack the received face data into the ghosts
    Riemann on every local face (partition faces on both sides), corrector
    dt = min over ranks of the local dt_next

and equals the unpartitioned step cell for cell.  Remeshing runs on every
rank with the same whole-mesh flags, then cells that change owner migrate.

This module only orders calls and moves buffers between ranks: the
arithmetic of every step runs in the library's kernels.  Two exchanges:
``LocalExchange`` for several sub-domains in one process (device copies
between their buffers), ``DistExchange`` for one sub-domain per process over
``torch.distributed`` (NCCL with device tensors, gloo through host copies).
"""

from . import ader as A


class SubDomain:
    """One rank's part of a partitioned mesh.  ``solver`` is a ``Solver``
    whose context holds the whole mesh and state; it is partitioned in place
    and keeps its owned rows of the state."""

    def __init__(self, solver, nranks, rank):
        self.solver = solver
        self.torch = solver.torch
        self.nranks, self.rank = nranks, rank
        A.ader_partition(solver.ctx, nranks, rank)
        self.dt_local = self.torch.zeros(1, dtype=self.torch.float64, device=solver.device)
        self._halo_buffers()

    @property
    def ctx(self):
        return self.solver.ctx

    def info(self):
        """(nranks, rank, nglobal, first, nowned, nghost)."""
        return A.ader_dd_info(self.ctx)

    def cuts(self):
        return A.ader_dd_cuts(self.ctx)

    def peers(self):
        return [p for p in range(self.nranks) if p != self.rank]

    def _buffer(self, n):
        return self.torch.empty(int(n), dtype=self.torch.float64, device=self.solver.device)

    def _halo_buffers(self):
        self.halo_send, self.halo_recv = {}, {}
        for p in self.peers():
            ns, nr = A.ader_halo_size(self.ctx, p)
            if ns:
                self.halo_send[p] = self._buffer(ns)
            if nr:
                self.halo_recv[p] = self._buffer(nr)

    def halo_bytes(self):
        """Bytes this rank sends per step."""
        return 8 * sum(b.numel() for b in self.halo_send.values())

    # ------------------------------------------------------------ step parts
    def begin_step(self, stream=None):
        """Skeleton predictor and the packing of every neighbour's face data."""
        s = self.solver
        s.predict(A.ADER_SKELETON, stream)
        st = s._stream(stream)
        for p, buf in self.halo_send.items():
            A.ader_halo_pack(self.ctx, p, buf, st)

    def predict_enclave(self, stream=None):
        self.solver.predict(A.ADER_ENCLAVE, stream)

    def finish_step(self, stream=None):
        """Unpack the received face data, solve every local face, correct the
        owned cells; the local next time step lands in ``dt_local``."""
        s = self.solver
        st = s._stream(stream)
        for p, buf in self.halo_recv.items():
            A.ader_halo_unpack(self.ctx, p, buf, st)
        s.riemann(A.ADER_ALL, stream)
        s.correct(self.dt_local, stream)

    # ---------------------------------------------------------------- remesh
    def remesh(self, flags):
        """Adapt with whole-mesh flags (identical on every rank); returns the
        migration buffers to send, keyed by peer."""
        A.ader_remesh(self.ctx, flags)
        st = self.solver._stream(None)
        sends, self.migrate_recv_sizes = {}, {}
        for p in self.peers():
            ns, nr = A.ader_migrate_size(self.ctx, p)
            if ns:
                buf = self._buffer(ns)
                A.ader_migrate_pack(self.ctx, p, buf, st)
                sends[p] = buf
            if nr:
                self.migrate_recv_sizes[p] = nr
        return sends

    def finish_migration(self, recvs):
        st = self.solver._stream(None)
        for p, buf in recvs.items():
            A.ader_migrate_unpack(self.ctx, p, buf, st)
        self._halo_buffers()


class LocalExchange:
    """Several sub-domains of one mesh in one process (one GPU): the packed
    buffers are copied device to device, in the order of the calls on the
    current stream."""

    def __init__(self, subs):
        self.subs = sorted(subs, key=lambda s: s.rank)

    def halo(self):
        for s in self.subs:
            for p, buf in s.halo_send.items():
                self.subs[p].halo_recv[s.rank].copy_(buf)

    def min_dt(self):
        torch = self.subs[0].torch
        dt = torch.stack([s.dt_local for s in self.subs]).min(dim=0).values
        for s in self.subs:
            s.solver.dt.copy_(dt)

    def migrate(self, sends):
        """sends[r] = the buffers rank r packed (peer -> buffer)."""
        for s in self.subs:
            recvs = {}
            for p in s.migrate_recv_sizes:
                recvs[p] = sends[p][s.rank]
            s.finish_migration(recvs)


class DistExchange:
    """One sub-domain per process over torch.distributed: point-to-point
    sends and receives of the packed buffers (device tensors with NCCL; host
    copies with gloo), and an all-reduce of the time step."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.host = dist.get_backend(group) == "gloo"

    def exchange(self, sends, recv_sizes, like):
        """Send sends[p] to every peer p and receive recv_sizes[q] doubles
        from every peer q; returns {q: tensor} on the device of ``like``."""
        torch = __import__("torch")
        if like.is_cuda and self.host:
            torch.cuda.current_stream(like.device).synchronize()
        out = {q: torch.empty(int(n), dtype=torch.float64,
                              device="cpu" if self.host else like.device)
               for q, n in recv_sizes.items()}
        # one group of point-to-point operations: NCCL runs ungrouped sends and
        # receives in issue order, which can deadlock when two ranks both
        # receive first
        ops = [self.dist.P2POp(self.dist.irecv, out[q], q, self.group) for q in sorted(out)]
        ops += [self.dist.P2POp(self.dist.isend, sends[p].cpu() if self.host else sends[p], p,
                                self.group) for p in sorted(sends)]
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()
        if self.host and like.is_cuda:
            out = {q: t.to(like.device) for q, t in out.items()}
        return out

    def halo(self, sub):
        recvs = self.exchange(sub.halo_send, {q: b.numel() for q, b in sub.halo_recv.items()},
                              sub.dt_local)
        for q, t in recvs.items():
            if t is not sub.halo_recv[q]:
                sub.halo_recv[q].copy_(t)

    def min_dt(self, sub):
        v = sub.dt_local.cpu() if self.host else sub.dt_local.clone()
        self.dist.all_reduce(v, op=self.dist.ReduceOp.MIN, group=self.group)
        sub.solver.dt.copy_(v.to(sub.solver.device))

    def migrate(self, sub, sends):
        recvs = self.exchange(sends, sub.migrate_recv_sizes, sub.dt_local)
        sub.finish_migration(recvs)


def step_local(subs, exchange, nsteps=1):
    """nsteps steps of all sub-domains of one process (LocalExchange)."""
    for _ in range(nsteps):
        for s in subs:
            s.begin_step()
        for s in subs:
            s.predict_enclave()
        exchange.halo()
        for s in subs:
            s.finish_step()
        exchange.min_dt()


def remesh_local(subs, exchange, flags):
    sends = {s.rank: s.remesh(flags) for s in subs}
    exchange.migrate(sends)


def step_dist(sub, exchange, nsteps=1):
    """nsteps steps of this process's sub-domain (DistExchange); the enclave
    predictor is enqueued before the exchange waits, so on the GPU it runs
    while the face data travel."""
    for _ in range(nsteps):
        sub.begin_step()
        sub.predict_enclave()
        exchange.halo(sub)
        sub.finish_step()
        exchange.min_dt(sub)


def remesh_dist(sub, exchange, flags):
    exchange.migrate(sub, sub.remesh(flags))
