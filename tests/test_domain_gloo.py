"""Domain decomposition on CPU ranks (gloo, world sizes 2 and 3).

The partition and exchange lists come from the library's host partitioner
(ader_mesh_partition, the code the device sub-domains use), the buffers
travel through the driver's DistExchange, and each rank computes its part of
the step with the oracle's cell-local tasks: the predictor on its owned
cells, Rusanov (with prolongation and restriction) on every local face, the
corrector on its owned cells, and dt as the minimum over ranks.  Every rank
checks its owned cells against the oracle's whole-mesh step, over three
steps, a remesh with a new partition, and two more steps."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def local_riemann(part, Q, F, P, B, dim):
    """F* on the sub-domain's local faces (local cell numbering), with the
    oracle's Rusanov flux and face prolongation/restriction."""
    from oracle import ader
    from oracle.mesh import subface_indices
    Fs = np.full_like(Q, np.nan)
    conf = part["conf"]
    for dr in range(dim):
        sel = conf[conf[:, 2] == dr]
        if len(sel):
            cL, cR = sel[:, 0], sel[:, 1]
            Fstar = ader.rusanov(Q[cL, dr, 1], F[cL, dr, 1], Q[cR, dr, 0], F[cR, dr, 0], P, dr)
            Fs[cL, dr, 1] = Fstar
            Fs[cR, dr, 0] = Fstar
    par, kids = part["parents"], part["children"]
    for dr in range(dim):
        for cs in range(2):
            g = np.flatnonzero((par[:, 1] == dr) & (par[:, 2] == cs))
            if not len(g):
                continue
            coarse = par[g, 0]
            acc = np.zeros((len(g),) + Q.shape[3:])
            for j, s in enumerate(subface_indices(dim, dr)):
                fine = kids[g, j]
                Qv = ader.prolong_face(Q[coarse, dr, cs], s, B, dim)
                Fv = ader.prolong_face(F[coarse, dr, cs], s, B, dim)
                if cs == 1:
                    Fstar = ader.rusanov(Qv, Fv, Q[fine, dr, 0], F[fine, dr, 0], P, dr)
                    Fs[fine, dr, 0] = Fstar
                else:
                    Fstar = ader.rusanov(Q[fine, dr, 1], F[fine, dr, 1], Qv, Fv, P, dr)
                    Fs[fine, dr, 1] = Fstar
                acc += ader.restrict_face(Fstar, s, B, dim)
            Fs[coarse, dr, cs] = acc
    return Fs


def _pack(part, q, Q, F, dim):
    """The buffer for peer q: per exchange entry the slot's Q-bar then F-bar
    (the layout of the device pack kernel)."""
    ent = part["send"][part["send_off"][q]:part["send_off"][q + 1]]
    c, slot = ent // (2 * dim), ent % (2 * dim)
    blocks = [np.concatenate([Q[ci, sl // 2, sl % 2].ravel(), F[ci, sl // 2, sl % 2].ravel()])
              for ci, sl in zip(c, slot)]
    return np.concatenate(blocks) if blocks else np.zeros(0)


def _unpack(part, q, buf, Q, F, dim):
    ent = part["recv"][part["recv_off"][q]:part["recv_off"][q + 1]]
    blk = Q.shape[3] * Q.shape[4]
    for e, v in zip(ent, buf.reshape(len(ent), 2 * blk)):
        ci, sl = e // (2 * dim), e % (2 * dim)
        Q[ci, sl // 2, sl % 2] = v[:blk].reshape(Q.shape[3:])
        F[ci, sl // 2, sl % 2] = v[blk:].reshape(F.shape[3:])


def _worker(rank, world, port, dim, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, _run(rank, world, dim, torch, dist)))
    except Exception as e:  # report, do not hang the other ranks' queue reads
        import traceback
        out.put((rank, "".join(traceback.format_exception(e))))
    finally:
        dist.destroy_process_group()


def _run(rank, world, dim, torch, dist):
    from oracle import ader, basis, mesh as omesh, pde, step as ostep
    import workloads
    from paper_1806_07984_gb300 import ader as A
    from paper_1806_07984_gb300.domain import DistExchange
    order, base, levels = 2, (9 if dim == 2 else 4), (2 if dim == 2 else 1)
    B, P = basis.Basis(order), pde.Euler(dim)
    mesh = A.ader_mesh_create(dim, (base,) * dim, levels)
    om = omesh.Mesh(dim, (base,) * dim, levels)

    def keys():
        cells = A.ader_mesh_leaves(mesh)[0]
        return [(int(c[0]), tuple(int(x) for x in c[1:1 + dim])) for c in cells]

    def adapt(center, u):
        fo = omesh.sphere_flags(om, center, 0.22)
        perm = np.array([om.index[k] for k in keys()])
        A.ader_mesh_adapt(mesh, fo[perm])
        return om.remesh(u, fo, B)

    c0 = (0.4, 0.55, 0.5)[:dim]
    u = np.ones((len(om.cells), dim + 2) + (B.n,) * dim)
    for _ in range(levels):
        u = adapt(c0, u)
    X = om.node_coords(B.xi)
    u = np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X, sigma=0.12,
                                                                  center=(0.5,) * dim), 0, 1))
    cfl = workloads.ADER_CFL[order]
    dt = ader.cfl_dt(u, om.cell_widths(), P, order, cfl=cfl)
    ex = DistExchange()
    like = torch.zeros(1, dtype=torch.float64)
    checked = []
    for phase in range(2):
        perm = np.array([om.index[k] for k in keys()])
        part = A.ader_mesh_partition(mesh, world, rank, dim)
        first, nown = part["first"], part["nowned"]
        glob = np.concatenate([perm[first:first + nown], perm[part["ghosts"]]])  # local -> oracle
        h = om.cell_widths()[glob]
        u_own = u[perm[first:first + nown]].copy()
        for _ in range(3 if phase == 0 else 2):
            ustar, Qf, Ff = ostep.predict(u_own, h[:nown], dt, P, B, order + 1)
            shape = (len(glob),) + Qf.shape[1:]
            Q, F = np.full(shape, np.nan), np.full(shape, np.nan)
            Q[:nown], F[:nown] = Qf, Ff
            sends = {q: torch.from_numpy(_pack(part, q, Q, F, dim)) for q in range(world)
                     if q != rank and part["send_off"][q + 1] > part["send_off"][q]}
            blk2 = 2 * Q.shape[3] * Q.shape[4]
            sizes = {q: int(part["recv_off"][q + 1] - part["recv_off"][q]) * blk2
                     for q in range(world) if q != rank and part["recv_off"][q + 1] > part["recv_off"][q]}
            for q, t in ex.exchange(sends, sizes, like).items():
                _unpack(part, q, t.numpy(), Q, F, dim)
            Fs = local_riemann(part, Q, F, P, B, dim)
            u_own = ader.face_lifting(ustar, Fs[:nown], h[:nown], dt, B)
            dtl = torch.tensor([ader.cfl_dt(u_own, h[:nown], P, order, cfl=cfl)], dtype=torch.float64)
            dist.all_reduce(dtl, op=dist.ReduceOp.MIN)
            ref = ostep.step(om, u, dt, P, B)
            err = np.abs(u_own - ref.u[perm[first:first + nown]]).max() / np.abs(ref.u).max()
            checked.append((phase, float(err), float(dtl.item()), float(ref.dt_next),
                            int(part["nghost"]), int(len(part["parents"]))))
            u, dt = ref.u, float(dtl.item())
        u = adapt(tuple(x + 0.2 for x in c0), u)
        dt = ader.cfl_dt(u, om.cell_widths(), P, order, cfl=cfl)
    A.ader_mesh_destroy(mesh)
    return checked


@pytest.mark.parametrize("world,dim", [(2, 2), (3, 2), (3, 3)])
def test_partitioned_step_on_gloo_ranks(world, dim):
    import torch.multiprocessing as mp
    from paper_1806_07984_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, dim, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
    for rank in range(world):
        assert not isinstance(res[rank], str), res[rank]
        assert len(res[rank]) == 5
        for phase, err, dt_got, dt_ref, nghost, npar in res[rank]:
            assert err < 1e-13, (rank, phase, err)
            assert abs(dt_got - dt_ref) <= 1e-14 * dt_ref
            assert nghost > 0
    assert any(r[5] > 0 for v in res.values() for r in v)     # transitions inside sub-domains
    for p in procs:
        assert p.exitcode == 0
