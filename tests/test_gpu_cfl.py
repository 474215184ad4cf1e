"""The CFL reduction (global time stepping, Sec. 2.1) with its maximum on a
node owned by the last, partial warp of a CTA.

The rate kernels run one thread per spatial node and CPB cells per CTA, so a
CTA has CPB n^d threads: 216 at 3D N=5, 250 at 3D N=4, 252 at 2D N=5 and 243
at 3D N=2, each ending in a warp with fewer than 32 lanes.  One node in the
middle of that warp gets a pressure 60 times the background, so its wave
speed decides dt; the node carries the peak of a smooth pressure bump over
its cell, so that the face values stay physical.  ader_compute_dt, the
corrector's dt_next and the allocation-free ader_compute_dt_static must all
equal the oracle's dt = C / max sum_d lambda_d / h_d."""
import numpy as np
import pytest

from oracle import ader as oader, basis as obasis, pde as opde, step as ostep
import workloads
from gpu_helpers import build_pair, rel_l2
from oracle_helpers import random_state

pytestmark = pytest.mark.gpu

TOL = 1e-13
GAMMA = 1.4


def _shape(dim, order):
    NS = (order + 1) ** dim
    CPB = 1 if NS >= 128 else 256 // NS
    return NS, CPB, CPB * NS


def _hot_state(om, B, perm, dim, order, seed):
    """Random Euler state whose largest rate sits on a node that the CTA's
    last (partial) warp owns; returns the state and that (cell, node).

    The hot cell holds rho = 1, v = 0.5 and p = 1 + 59 (1 - |x - x_hot|^2 /
    L^2), L its diagonal: a quadratic, so every point of the cell, its faces
    included, keeps p >= 1, and since the rate there grows with p alone the
    nodal maximum is the node x_hot."""
    NS, CPB, threads = _shape(dim, order)
    assert threads % 32 != 0
    first = threads // 32 * 32
    tid = first + (threads - first) // 2          # a middle lane of the partial warp
    cl, node = divmod(tid, NS)
    cell = 2 * CPB + cl                           # third CTA of the launch
    assert cell < len(perm)
    u = random_state(om, B, "euler", seed)
    oc = perm[cell]
    X = om.node_coords(B.xi)
    xs = [X[d][oc].reshape(-1) for d in range(dim)]
    r2 = sum((xs[d] - xs[d][node]) ** 2 for d in range(dim))
    L2 = float(np.sum(om.cell_widths()[oc] ** 2))
    flat = u.reshape(u.shape[0], u.shape[1], -1)
    p = 1.0 + 59.0 * (1.0 - r2 / L2)
    flat[oc, 0] = 1.0
    flat[oc, 1:dim + 1] = 0.5
    flat[oc, dim + 1] = p / (GAMMA - 1.0) + 0.5 * dim * 0.25
    return u, cell, node


def _node_rates(u, h, P):
    """Per-node sum_d lambda_d / h_d, only to locate the maximum."""
    q = np.moveaxis(u.reshape(u.shape[0], u.shape[1], -1), 1, 0)
    return sum(P.max_speed(q, d) / h[:, d:d + 1] for d in range(h.shape[1]))


@pytest.mark.parametrize("dim,order,base", [(3, 5, 3), (3, 4, 3), (2, 5, 9), (3, 2, 3)])
def test_cfl_maximum_in_last_partial_warp(dim, order, base):
    import torch
    from paper_1806_07984_gb300 import ader as A
    solver, om, perm = build_pair(dim, order, "euler", base, 0)
    B = obasis.Basis(order)
    P = opde.Euler(dim)
    u0, cell, node = _hot_state(om, B, perm, dim, order, seed=60 + 10 * dim + order)
    h = om.cell_widths()
    cfl = workloads.ADER_CFL[order]
    dt = oader.cfl_dt(u0, h, P, order, cfl=cfl)
    # the hot node decides dt, by a clear margin over every other node
    rates = _node_rates(u0, h, P)
    assert np.unravel_index(np.argmax(rates), rates.shape) == (perm[cell], node)
    assert np.sort(rates.ravel())[-2] < (1 - 1e-3) * rates.max()

    solver.set_state(u0[perm])
    got = solver.compute_dt().item()
    assert abs(got - dt) <= TOL * dt, (got, dt)

    # allocation-free entry point on the same state
    cfg = solver.cfg
    lv = torch.from_numpy(solver.cells()[:, 0].astype(np.int8)).to(solver.device)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=solver.device)
    A.ader_compute_dt_static(cfg.dim, cfg.order, cfg.pde, cfg.gamma, cfg.cfl, list(cfg.base),
                             list(cfg.lo), list(cfg.hi), solver.ncells,
                             solver.get_state().data_ptr(), lv.data_ptr(), out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert abs(out.item() - dt) <= TOL * dt, (out.item(), dt)

    # corrector's dt_next: a short step keeps the maximum on the hot node
    dt_step = 1e-3 * dt
    ref = ostep.step(om, u0, dt_step, P, B)
    solver.set_dt(dt_step)
    solver.predict()
    solver.riemann()
    dt_next = solver.dt.clone()
    solver.correct(dt_next)
    u1 = solver.get_state().cpu().numpy()
    assert rel_l2(u1, ref.u[perm]) < 1e-12
    assert abs(dt_next.item() - ref.dt_next) <= TOL * ref.dt_next, (dt_next.item(), ref.dt_next)
    assert solver.status() == 0
    solver.close()
