"""Discrete adjoint of the linear-acoustics step: against the transpose of
the oracle's step matrix, the dot-product identity on the full 27^3 N=4
mesh, and the misfit gradient against central finite differences."""
import numpy as np
import pytest

from oracle import ader as oader, basis as obasis, mesh as omesh, pde as opde, step as ostep
import workloads
from gpu_helpers import lib_keys, rel_l2

pytestmark = pytest.mark.gpu


def solver_for(dim, order, base, iters, predictor="picard", max_level=0):
    from paper_1806_07984_gb300 import Solver
    return Solver(dim, order, "acoustics", base=(base,) * 3, max_level=max_level,
                  cfl=workloads.ADER_CFL[order], picard_iters=iters, predictor=predictor)


def amr_pair(dim, order, base, iters, predictor, center, radius, levels=1):
    """Library context and oracle mesh refined the same way around a ball."""
    s = solver_for(dim, order, base, iters, predictor, max_level=levels)
    m = omesh.Mesh(dim, (base,) * dim, levels)
    for _ in range(levels):
        fl = omesh.sphere_flags(m, center, radius)
        s.remesh(fl[np.array([m.index[k] for k in lib_keys(s)])])
        m.remesh(np.zeros((len(m.cells), 1) + (2,) * dim), fl, obasis.Basis(1))
    assert sorted(lib_keys(s)) == m.cells
    return s, m


# uniform meshes, and meshes with one refined region (resolution transitions:
# the adjoint of the prolongation, child-face Rusanov and restriction)
@pytest.mark.parametrize("dim,order,base,predictor,amr", [
    (3, 2, 2, "picard", False), (2, 3, 3, "picard", False), (3, 2, 2, "ck", False),
    (2, 4, 3, "ck", False), (2, 2, 3, "picard", True), (2, 3, 3, "ck", True),
    (3, 1, 3, "picard", True)])
def test_adjoint_equals_transpose_of_oracle_step(dim, order, base, predictor, amr):
    import torch
    from paper_1806_07984_gb300 import ader as A
    iters = dim * order + 1
    if amr:
        s, m = amr_pair(dim, order, base, iters, predictor, (0.5, 0.5, 0.5)[:dim], 0.1)
        assert s.mesh_info()[3] > 0
    else:
        s = solver_for(dim, order, base, iters, predictor)
        m = omesh.Mesh(dim, (base,) * dim, 0)
    perm = np.array([m.index[k] for k in lib_keys(s)])
    B = obasis.Basis(order)
    P = opde.Acoustics(dim)
    shape = (len(m.cells), dim + 1) + (B.n,) * dim
    dt = workloads.ADER_CFL[order] / (dim * base * (3 if amr else 1))
    size = int(np.prod(shape))
    Amat = np.zeros((size, size))
    for j in range(size):
        e = np.zeros(size)
        e[j] = 1.0
        Amat[:, j] = ostep.step(m, e.reshape(shape), dt, P, B, iters=iters,
                                predictor=predictor).u.ravel()
    rng = np.random.default_rng(1)
    y = rng.standard_normal(shape)
    ref = (Amat.T @ y.ravel()).reshape(shape)          # oracle order
    lam_in = torch.from_numpy(np.ascontiguousarray(y[perm])).cuda()
    lam_out = torch.empty_like(lam_in)
    s.set_dt(dt)
    A.ader_adjoint_step(s.ctx, lam_in, lam_out, s.dt)
    torch.cuda.synchronize()
    assert rel_l2(lam_out.cpu().numpy(), ref[perm]) < 1e-12
    # the forward step is the oracle's matrix too
    x = rng.standard_normal(shape)
    s.set_state(np.ascontiguousarray(x[perm]))
    s.set_dt(dt)
    s.predict(); s.riemann(); s.correct(torch.zeros_like(s.dt))
    fwd = s.get_state().cpu().numpy()
    assert rel_l2(fwd, (Amat @ x.ravel()).reshape(shape)[perm]) < 1e-12
    s.close()


@pytest.fixture(scope="module")
def cfg5():
    """3D acoustics N=4 on 27^3, Picard dN+1 = 13 iterations, fixed dt."""
    import torch
    order, base = 4, 27
    s = solver_for(3, order, base, 3 * order + 1)
    X = s.node_coords()
    u0 = torch.from_numpy(np.ascontiguousarray(
        np.moveaxis(workloads.acoustic_pulses(X, seed=1), 0, 1))).cuda()
    uobs = torch.from_numpy(np.ascontiguousarray(
        np.moveaxis(workloads.acoustic_pulses(X, seed=3), 0, 1))).cuda()
    s.set_state(u0)
    s.compute_dt()
    dt = s.dt.clone()
    return s, u0, uobs, dt


def test_dot_product_identity_full_mesh(cfg5):
    import torch
    from paper_1806_07984_gb300 import ader as A
    s, u0, _, dt = cfg5
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(u0.shape, dtype=torch.float64, device="cuda", generator=g)
    y = torch.randn(u0.shape, dtype=torch.float64, device="cuda", generator=g)
    s.set_state(x)
    s.dt.copy_(dt)
    s.predict(); s.riemann(); s.correct(torch.zeros_like(dt))
    Ax = s.get_state()
    Aty = torch.empty_like(y)
    A.ader_adjoint_step(s.ctx, y, Aty, dt)
    lhs = float((Ax * y).sum())
    rhs = float((x * Aty).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), float(Ax.norm() * y.norm()) * 1e-3)


def test_misfit_gradient_vs_central_differences(cfg5):
    import torch
    from paper_1806_07984_gb300 import adjoint as adj
    s, u0, uobs, dt = cfg5
    rec = adj.Receivers(s, workloads.acoustic_receivers(64, seed=2))
    nsteps = 50
    p_obs, _ = adj.forward_run(s, uobs, dt, rec, nsteps)
    loss_fn = adj.AcousticMisfit.make(s, dt, rec, p_obs, nsteps, every=10)
    u = u0.clone().requires_grad_(True)
    loss = loss_fn(u)
    loss.backward()
    grad = u.grad
    assert float(loss) > 0 and torch.isfinite(grad).all()
    h = 1e-6
    g = torch.Generator(device="cuda").manual_seed(8)
    for k in range(8):
        v = torch.randn(u0.shape, dtype=torch.float64, device="cuda", generator=g)
        lp, _ = adj.misfit(s, u0 + h * v, dt, rec, p_obs, nsteps)
        lm, _ = adj.misfit(s, u0 - h * v, dt, rec, p_obs, nsteps)
        fd = (lp - lm) / (2 * h)
        an = float((grad * v).sum())
        assert abs(fd - an) <= 1e-5 * abs(an), (k, fd, an)


def test_ck_gradient_vs_central_differences():
    """The misfit gradient with the Cauchy-Kowalevski predictor (27^3, N=4)."""
    import torch
    from paper_1806_07984_gb300 import adjoint as adj
    s = solver_for(3, 4, 27, 0, "ck")
    X = s.node_coords()
    u0 = torch.from_numpy(np.ascontiguousarray(
        np.moveaxis(workloads.acoustic_pulses(X, seed=1), 0, 1))).cuda()
    uobs = torch.from_numpy(np.ascontiguousarray(
        np.moveaxis(workloads.acoustic_pulses(X, seed=3), 0, 1))).cuda()
    s.set_state(u0)
    s.compute_dt()
    dt = s.dt.clone()
    rec = adj.Receivers(s, workloads.acoustic_receivers(64, seed=2))
    nsteps = 50
    p_obs, _ = adj.forward_run(s, uobs, dt, rec, nsteps)
    loss_fn = adj.AcousticMisfit.make(s, dt, rec, p_obs, nsteps, every=10)
    u = u0.clone().requires_grad_(True)
    loss_fn(u).backward()
    g = torch.Generator(device="cuda").manual_seed(8)
    for k in range(4):
        v = torch.randn(u0.shape, dtype=torch.float64, device="cuda", generator=g)
        lp, _ = adj.misfit(s, u0 + 1e-6 * v, dt, rec, p_obs, nsteps)
        lm, _ = adj.misfit(s, u0 - 1e-6 * v, dt, rec, p_obs, nsteps)
        fd = (lp - lm) / 2e-6
        an = float((u.grad * v).sum())
        assert abs(fd - an) <= 1e-5 * abs(an), (k, fd, an)
    s.close()


@pytest.mark.parametrize("predictor", ["picard", "ck"])
def test_dot_product_identity_amr_mesh(predictor):
    """<A x, y> = <x, A^T y> on a 3D N=4 acoustics mesh with two levels of
    refinement around a ball (hanging faces on both levels)."""
    import torch
    from paper_1806_07984_gb300 import ader as A
    order = 4
    s, m = amr_pair(3, order, 9, 3 * order + 1, predictor, (0.45, 0.5, 0.55), 0.15, levels=2)
    assert s.mesh_info()[3] > 0
    shape = s.state_shape()
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(shape, dtype=torch.float64, device="cuda", generator=g)
    y = torch.randn(shape, dtype=torch.float64, device="cuda", generator=g)
    s.set_state(x)
    s.compute_dt()
    dt = s.dt.clone()
    s.predict(); s.riemann(); s.correct(torch.zeros_like(dt))
    Ax = s.get_state()
    Aty = torch.empty_like(y)
    A.ader_adjoint_step(s.ctx, y, Aty, dt)
    lhs = float((Ax * y).sum())
    rhs = float((x * Aty).sum())
    assert abs(lhs - rhs) <= 1e-12 * float(Ax.norm() * y.norm())
    s.close()
