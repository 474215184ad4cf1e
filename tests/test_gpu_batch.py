"""Batched instances (one CUDA graph of persistent phase kernels) against the
oracle run instance by instance."""
import numpy as np
import pytest

from oracle import ader as oader, basis as obasis, mesh as omesh, pde as opde, step as ostep
import workloads
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

INSTANCES = [(3, 1), (4, 2), (5, 3), (4, 4), (3, 5), (2, 6), (3, 7), (6, 3), (1, 2), (7, 5)]


def instance_state(side, order, center, eps, R=0.15):
    """Oracle-layout state of a vortex instance and the permutation from the
    batch cell order (x fastest) to the oracle's cell order."""
    m = omesh.Mesh(2, (side, side), 0)
    B = obasis.Basis(order)
    X = m.node_coords(B.xi)
    u = np.ascontiguousarray(np.moveaxis(
        workloads.isentropic_vortex(X[0], X[1], center=center, eps=eps, R=R), 0, 1))
    perm = np.array([m.index[(0, (c % side, c // side))] for c in range(side * side)])
    return m, B, u, perm


def make_batch(precision):
    from paper_1806_07984_gb300 import ader as A
    cfg = A.ader_batch_config()
    cfg.dim, cfg.pde, cfg.gamma, cfg.picard_iters = 2, A.ADER_EULER, 1.4, 0
    cfg.prec = A.ADER_FP64 if precision == "fp64" else A.ADER_FP32
    sides = [s for s, _ in INSTANCES]
    orders = [o for _, o in INSTANCES]
    cfls = [workloads.ADER_CFL[o] for o in orders]
    return A, A.ader_batch_init(cfg, sides, orders, cfls)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_batch_matches_oracle(precision, tol):
    import torch
    A, b = make_batch(precision)
    rng = np.random.default_rng(3)
    per = []
    for side, order in INSTANCES:
        center = tuple(rng.uniform(0, 1, 2))
        per.append(instance_state(side, order, center, float(rng.uniform(1, 5))))
    off = A.ader_batch_offsets(b, len(INSTANCES))
    u_all = np.concatenate([u[perm].ravel() for (_, _, u, perm) in per])
    assert len(u_all) == off[-1]
    u_dev = torch.from_numpy(u_all).cuda()
    A.ader_batch_set_state(b, u_dev.data_ptr(), True)
    A.ader_batch_compute_dt(b)
    dt0 = A.ader_batch_get_dt(b, len(INSTANCES))
    # autotuner: must leave state and dt untouched
    bps, tile, ms = A.ader_batch_tune(b)
    assert bps >= 1 and tile in (1, 2, 4, 8) and ms > 0
    back = torch.empty_like(u_dev)
    A.ader_batch_get_state(b, back.data_ptr(), True)
    torch.cuda.synchronize()
    assert torch.equal(back, u_dev)
    assert np.array_equal(A.ader_batch_get_dt(b, len(INSTANCES)), dt0)
    nsteps = 3
    A.ader_batch_run(b, nsteps)
    got = torch.empty_like(u_dev)
    A.ader_batch_get_state(b, got.data_ptr(), True)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    dts = A.ader_batch_get_dt(b, len(INSTANCES))
    assert A.ader_batch_status_word(b) == 0
    P = opde.Euler(2)
    for i, ((side, order), (m, B, u, perm)) in enumerate(zip(INSTANCES, per)):
        h = m.cell_widths()
        dt = oader.cfl_dt(u, h, P, order, cfl=workloads.ADER_CFL[order])
        assert abs(dt0[i] - dt) <= 1e-13 * dt
        for _ in range(nsteps):
            out = ostep.step(m, u, dt, P, B)
            u, dt = out.u, out.dt_next
        mine = got[off[i]:off[i + 1]].reshape(u.shape)
        assert rel_l2(mine, u[perm]) < tol, (i, side, order, rel_l2(mine, u[perm]))
        assert abs(dts[i] - dt) <= max(tol, 1e-13) * dt * 10
    A.ader_batch_destroy(b)


def test_batch_graph_reuse_and_launch_shapes():
    """Two runs of 2 steps equal one run of 4 steps, whatever the launch shape."""
    import torch
    A, b = make_batch("fp64")
    rng = np.random.default_rng(9)
    parts = []
    for s, o in INSTANCES:
        _, _, u, perm = instance_state(s, o, tuple(rng.uniform(0, 1, 2)), 3.0)
        parts.append(u[perm].ravel())
    u_all = np.concatenate(parts)
    u_dev = torch.from_numpy(u_all).cuda()
    results = []
    for shape, runs in (((1, 1), (4,)), ((1, 8), (2, 2)), ((1, 4), (1, 3))):
        A.ader_batch_set_launch(b, *shape)
        A.ader_batch_set_state(b, u_dev.data_ptr(), True)
        A.ader_batch_compute_dt(b)
        for k in runs:
            A.ader_batch_run(b, k)
        got = torch.empty_like(u_dev)
        A.ader_batch_get_state(b, got.data_ptr(), True)
        torch.cuda.synchronize()
        results.append(got.cpu().numpy())
    assert A.ader_batch_status_word(b) == 0
    for r in results[1:]:
        assert rel_l2(r, results[0]) < 1e-14
    A.ader_batch_destroy(b)


def test_full_batch_sampled_instances():
    """The 512-instance batch of the bench (seed 0: sides 9..81, orders 3..7,
    1.4e6 cells) at the launch shape its autotuner picks, three steps in one
    graph launch; sampled instances -- the first three order-7 instances of
    side 27..45 and the first instance of side 27..45 of each other order
    (the oracle takes about 1 s per 81^2 cell-steps at N=7) -- equal the
    oracle run instance by instance, and all instances conserve mass."""
    import torch
    from paper_1806_07984_gb300 import ader as A
    specs = workloads.batch_instances(512, seed=0)
    sides = [sp["side"] for sp in specs]
    orders = [sp["order"] for sp in specs]
    cfg = A.ader_batch_config()
    cfg.dim, cfg.pde, cfg.gamma, cfg.picard_iters = 2, A.ADER_EULER, workloads.GAMMA, 0
    cfg.prec = A.ADER_FP64
    b = A.ader_batch_init(cfg, sides, orders, [workloads.ADER_CFL[o] for o in orders])
    parts, per = [], {}
    mid = [i for i, sp in enumerate(specs) if 27 <= sp["side"] <= 45]
    pick = [i for i in mid if specs[i]["order"] == 7][:3]
    for o in (3, 4, 5, 6):
        pick.append(next(i for i in mid if specs[i]["order"] == o))
    pick = sorted(set(pick))
    assert len(pick) == 7
    for i, sp in enumerate(specs):
        m, B, u, perm = instance_state(sp["side"], sp["order"], sp["center"], sp["eps"], R=0.1)
        parts.append(u[perm].ravel())
        if i in pick:
            per[i] = (m, B, u, perm)
    off = A.ader_batch_offsets(b, len(specs))
    u_dev = torch.from_numpy(np.concatenate(parts)).cuda()
    del parts
    A.ader_batch_set_state(b, u_dev.data_ptr(), True)
    A.ader_batch_compute_dt(b)
    bps, tile, ms = A.ader_batch_tune(b)
    assert bps >= 1 and tile in (1, 2, 4, 8)
    nsteps = 3
    A.ader_batch_run(b, nsteps)
    got = torch.empty_like(u_dev)
    A.ader_batch_get_state(b, got.data_ptr(), True)
    torch.cuda.synchronize()
    assert A.ader_batch_status_word(b) == 0
    dts = A.ader_batch_get_dt(b, len(specs))
    got = got.cpu().numpy()
    P = opde.Euler(2)
    for i in pick:
        m, B, u, perm = per[i]
        order = specs[i]["order"]
        h = m.cell_widths()
        dt = oader.cfl_dt(u, h, P, order, cfl=workloads.ADER_CFL[order])
        for _ in range(nsteps):
            out = ostep.step(m, u, dt, P, B)
            u, dt = out.u, out.dt_next
        mine = got[off[i]:off[i + 1]].reshape(u.shape)
        assert rel_l2(mine, u[perm]) < 1e-12, (i, specs[i], rel_l2(mine, u[perm]))
        assert np.abs(mine - u[perm]).max() <= 1e-11 * np.abs(u).max()
        assert abs(dts[i] - dt) <= 1e-12 * dt
    # mass of every instance is conserved (periodic squares)
    u0 = u_dev.cpu().numpy()
    for i, sp in enumerate(specs):
        n = sp["order"] + 1
        w = np.polynomial.legendre.leggauss(n)[1] / 2.0
        W = np.outer(w, w).ravel()
        r0 = u0[off[i]:off[i + 1]].reshape(sp["side"] ** 2, 4, n * n)[:, 0] @ W
        r1 = got[off[i]:off[i + 1]].reshape(sp["side"] ** 2, 4, n * n)[:, 0] @ W
        assert abs(r1.sum() - r0.sum()) <= 1e-12 * r0.sum()
    A.ader_batch_destroy(b)
