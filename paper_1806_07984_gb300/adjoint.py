"""Receiver misfit of a linear-acoustics ADER-DG run and its gradient with
respect to the initial state, through the library's hand-written discrete
adjoint (ader_adjoint_step), behind a torch.autograd.Function.

The forward run keeps a checkpoint of the state every `every` steps; the
backward pass recomputes each segment's states from its checkpoint (forward
steps on the device), re-evaluates the receiver residuals there, and sweeps
the adjoint state back through the segment:

    L = 1/2 sum_{n=1..N} sum_r (p_r(u^n) - p_obs[n, r])^2,   u^n = A u^(n-1)
    dL/du^0 = sum_n (A^T)^n S^T r_n,   lambda <- A^T (lambda + S^T r_n), n = N..1

where S samples the pressure at the receivers (Lagrange basis of the
containing cell at each receiver) and A is one step with the fixed dt.
"""
import numpy as np

from . import ader as A


def lagrange_row(nodes, x):
    """phi_j(x) for the Lagrange basis on `nodes` (product formula)."""
    n = len(nodes)
    out = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                out[j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return out


def receiver_weights(solver, points):
    """Containing cell and node weights (Lagrange basis at the reference
    coordinates) of every point; node index with x fastest."""
    cells = solver.cells()
    xi = solver.nodes()
    dim, n = solver.dim, solver.n
    lo = np.array(solver.cfg.lo[:dim])
    hi = np.array(solver.cfg.hi[:dim])
    base = np.array(solver.cfg.base[:dim], dtype=np.float64)
    h = (hi - lo)[None, :] / (base[None, :] * 3.0 ** cells[:, :1])
    org = lo[None, :] + cells[:, 1:1 + dim] * h
    idx = np.zeros(len(points), dtype=np.int32)
    W = np.zeros((len(points), n ** dim))
    for p, x in enumerate(np.asarray(points, dtype=np.float64)):
        inside = np.all((x[None, :] >= org) & (x[None, :] < org + h), axis=1)
        c = int(np.flatnonzero(inside)[0])
        ref = (x - org[c]) / h[c]
        rows = [lagrange_row(xi, ref[d]) for d in range(dim)]
        w = rows[0]
        for d in range(1, dim):
            w = np.multiply.outer(rows[d], w)     # slower directions first
        idx[p] = c
        W[p] = w.ravel()
    return idx, W


class Receivers:
    """Device copies of the receiver cells and weights for one solver."""

    def __init__(self, solver, points, var=0):
        import torch
        idx, W = receiver_weights(solver, points)
        self.n = len(points)
        self.var = var
        self.cells = torch.from_numpy(idx).to(solver.device)
        self.weights = torch.from_numpy(W).to(solver.device)

    def sample(self, solver, field, out):
        A.ader_sample(solver.ctx, self.n, self.cells, self.weights, self.var, field, out,
                      solver._stream(None))

    def sample_adjoint(self, solver, values, field):
        A.ader_sample_adjoint(solver.ctx, self.n, self.cells, self.weights, self.var, values,
                              field, solver._stream(None))


def step_fixed_dt(solver, dt_dev, dt_scratch):
    """One forward step with a fixed dt (the CFL update goes to a scratch)."""
    solver.dt.copy_(dt_dev)
    solver.predict()
    solver.riemann()
    solver.correct(dt_scratch)


def forward_run(solver, u0, dt_dev, receivers, nsteps, every=0):
    """Run nsteps from u0 (device tensor); returns receiver traces
    (nsteps, npts) and the checkpoints {step: state} every `every` steps."""
    import torch
    solver.set_state(u0)
    scratch = torch.zeros_like(dt_dev)
    traces = torch.zeros((nsteps, receivers.n), dtype=torch.float64, device=u0.device)
    ckpt = {}
    for k in range(nsteps):
        if every and k % every == 0:
            ckpt[k] = solver.get_state()
        step_fixed_dt(solver, dt_dev, scratch)
        receivers.sample(solver, None, traces[k])
    return traces, ckpt


def backward_sweep(solver, ckpt, dt_dev, receivers, p_obs, nsteps, every, scale=1.0):
    """dL/du0 (times `scale`) from the checkpoints of a forward run:
    recompute each segment from its checkpoint, then sweep the adjoint."""
    import torch
    u_like = ckpt[0]
    lam = torch.zeros_like(u_like)
    tmp = torch.zeros_like(u_like)
    scratch = torch.zeros_like(dt_dev)
    for s0 in reversed(sorted(ckpt)):
        s1 = min(s0 + every, nsteps)
        solver.set_state(ckpt[s0])
        seg_res = torch.zeros((s1 - s0, receivers.n), dtype=torch.float64, device=u_like.device)
        for j in range(s1 - s0):
            step_fixed_dt(solver, dt_dev, scratch)
            receivers.sample(solver, None, seg_res[j])
        seg_res = (seg_res - p_obs[s0:s1]) * scale
        for n in range(s1, s0, -1):
            receivers.sample_adjoint(solver, seg_res[n - s0 - 1].contiguous(), lam)
            A.ader_adjoint_step(solver.ctx, lam, tmp, dt_dev, solver._stream(None))
            lam, tmp = tmp, lam
    return lam


def misfit(solver, u0, dt_dev, receivers, p_obs, nsteps, every=0):
    """Loss of a forward run (and its checkpoints)."""
    traces, ckpt = forward_run(solver, u0, dt_dev, receivers, nsteps, every)
    res = traces - p_obs
    return 0.5 * float((res * res).sum()), ckpt


def misfit_and_gradient(solver, u0, dt_dev, receivers, p_obs, nsteps, every=10):
    """Loss and dL/du0 with checkpointed recomputation."""
    loss, ckpt = misfit(solver, u0, dt_dev, receivers, p_obs, nsteps, every)
    return loss, backward_sweep(solver, ckpt, dt_dev, receivers, p_obs, nsteps, every)


class AcousticMisfit:
    """torch.autograd.Function factory: loss(u0); backward runs the library's
    discrete adjoint with checkpointed recomputation."""

    @staticmethod
    def make(solver, dt_dev, receivers, p_obs, nsteps, every=10):
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, u0):
                loss, ckpt = misfit(solver, u0.detach().contiguous(), dt_dev, receivers, p_obs,
                                    nsteps, every)
                ctx.ckpt = ckpt
                return torch.tensor(loss, dtype=torch.float64, device=u0.device)

            @staticmethod
            def backward(ctx, g):
                grad = backward_sweep(solver, ctx.ckpt, dt_dev, receivers, p_obs, nsteps, every)
                ctx.ckpt = None
                return g * grad

        return _F.apply
