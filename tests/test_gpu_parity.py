"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on
identical seeded inputs.  FP64 bar: relative L2 <= 1e-12 per field (the
spec tolerance); FP32-predictor bar: relative L2 <= 1e-6."""
import numpy as np
import pytest

from oracle import ader as oader, basis as obasis, mesh as omesh, pde as opde, step as ostep
import workloads
from gpu_helpers import build_pair, close_fields, lib_keys, rel_l2
from oracle_helpers import random_state, state_from

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


def _tf32(x):
    """Round to TF32 (10 stored mantissa bits, nearest with ties away from
    zero, the rounding the kernel applies to its tensor-core operands) after
    rounding to FP32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    b = (b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return b.view(np.float32).astype(np.float64)


def tf32_operand_tolerance(om, u0, dt, P, B, factor=4.0):
    """Bounds for the plain-TF32 predictor derived from its operand rounding:
    the oracle's step with the predictor's derivative operator D/h rounded to
    TF32 per level (what the tensor cores multiply by), against the exact
    step.  The kernel also rounds the fluxes (the other operand, an error of
    the same statistical size), so the bound is `factor` (4) times the
    relative change, for the fields and for the increments."""
    from types import SimpleNamespace
    h = om.cell_widths()
    ref = ostep.step(om, u0, dt, P, B)
    q = np.empty((len(u0), B.n) + u0.shape[1:])
    for hv in np.unique(h[:, 0]):
        sel = np.flatnonzero(h[:, 0] == hv)
        Bp = SimpleNamespace(n=B.n, phi0=B.phi0, w=B.w, K1=B.K1, D=_tf32(B.D / hv) * hv)
        q[sel] = oader.picard_predictor(u0[sel], h[sel], dt, P, Bp, B.order + 1)
    qbar, fbar = oader.time_average(q, P, B)
    ustar = oader.volume_update(u0, fbar, h, dt, B)
    Qf, Ff = oader.project_to_faces(qbar, fbar, B)
    Fs = ostep.riemann(om, Qf, Ff, P, B)
    u1, _ = ostep.correct(ustar, Fs, h, dt, P, B)
    fields = max(rel_l2(ustar, ref.ustar), rel_l2(Qf, ref.Qf), rel_l2(Ff, ref.Ff),
                 rel_l2(Fs, ref.Fs), rel_l2(u1, ref.u))
    incs = max(rel_l2(ustar - u0, ref.ustar - u0), rel_l2(u1 - u0, ref.u - u0))
    assert fields > 0 and incs > 0
    return factor * fields, factor * incs


def stage_parity(dim, order, pde, base, max_level, centers, radius, seed, tol=TOL64,
                 precision="fp64", predictor="picard", tol_from=None):
    import paper_1806_07984_gb300.ader as A
    solver, om, perm = build_pair(dim, order, pde, base, max_level, centers, radius,
                                  precision=precision, predictor=predictor)
    B = obasis.Basis(order)
    P = opde.make_pde(pde, dim)
    u0 = random_state(om, B, pde, seed)
    h = om.cell_widths()
    dt = oader.cfl_dt(u0, h, P, order, cfl=workloads.ADER_CFL[order])
    ref = ostep.step(om, u0, dt, P, B, predictor=predictor)
    tol_inc = max(tol * 1e3, 1e-9)
    if tol_from is not None:
        tol, tol_inc = tol_from(om, u0, dt, P, B)
    solver.set_state(u0[perm])
    solver.set_dt(dt)
    solver.predict()
    ustar = solver.get_field(A.ADER_FIELD_USTAR).cpu().numpy()
    fq = solver.get_field(A.ADER_FIELD_FACE_Q).cpu().numpy()
    ff = solver.get_field(A.ADER_FIELD_FACE_F).cpu().numpy()
    # every field by relative L2 <= tol and element by element <= 10 tol
    assert close_fields(ustar - u0[perm], ref.ustar[perm] - u0[perm], tol_inc)
    assert close_fields(ustar, ref.ustar[perm], tol)
    assert close_fields(fq, ref.Qf[perm], tol)
    assert close_fields(ff, ref.Ff[perm], tol)
    solver.riemann()
    fs = solver.get_field(A.ADER_FIELD_FSTAR).cpu().numpy()
    assert close_fields(fs, ref.Fs[perm], tol)
    dt_next = solver.dt.clone()
    solver.correct(dt_next)
    u1 = solver.get_state().cpu().numpy()
    assert close_fields(u1 - u0[perm], ref.u[perm] - u0[perm], tol_inc)
    assert close_fields(u1, ref.u[perm], tol)
    assert abs(dt_next.item() - ref.dt_next) < tol * ref.dt_next
    # conservation on the periodic mesh holds to FP64 rounding in every precision
    I0 = oader.cell_integral(u0, h, B)
    I1 = oader.cell_integral(u1, h[perm], B)
    assert np.allclose(I1, I0, rtol=0, atol=1e-13 * max(1.0, np.abs(I0).max())), I1 - I0
    assert solver.status() == 0
    n = solver.mesh_info()
    solver.close()
    return n


@pytest.mark.parametrize("order", [1, 3, 5, 7])
def test_uniform_2d_euler_stages(order):
    # 7 x 7 = 49 cells: not a multiple of the cells per CTA (ragged tail)
    n = stage_parity(2, order, "euler", 7, 0, (), 0.1, seed=order)
    assert n[3] == 0


@pytest.mark.parametrize("order", [2, 3, 5])
def test_amr_2d_euler_stages(order):
    n = stage_parity(2, order, "euler", 9, 2, [(0.45, 0.55)] * 2, 0.15, seed=10 + order)
    assert n[3] > 0 and n[1] > 0


@pytest.mark.parametrize("order", [2, 3, 5])
def test_amr_3d_euler_stages(order):
    n = stage_parity(3, order, "euler", 3, 2, [(0.45, 0.5, 0.55)] * 2, 0.12, seed=20 + order)
    assert n[3] > 0


@pytest.mark.parametrize("dim,order", [(2, 4), (3, 4)])
def test_amr_acoustics_stages(dim, order):
    c = (0.45, 0.5, 0.55)[:dim]
    stage_parity(dim, order, "acoustics", 3 if dim == 3 else 9, 2, [c] * 2, 0.12, seed=30 + dim)


@pytest.mark.parametrize("order", [3, 5])
def test_fp32_predictor_bound(order):
    stage_parity(3, order, "euler", 3, 1, [(0.5, 0.5, 0.5)], 0.2, seed=40, tol=TOL32,
                 precision="fp32")


def test_single_cell_self_periodic_3d():
    stage_parity(3, 3, "euler", 1, 0, (), 0.1, seed=50)


def test_3d_order7_fp64():
    stage_parity(3, 7, "euler", 2, 0, (), 0.1, seed=51)


def test_streams_step_matches_oracle_sequence():
    """ader_step on the two prioritised streams, dt kept on the device, three
    steps, against three oracle steps with the oracle's own dt sequence."""
    dim, order = 2, 3
    solver, om, perm = build_pair(dim, order, "euler", 9, 2, [(0.4, 0.6)] * 2, 0.15)
    B = obasis.Basis(order)
    P = opde.Euler(dim)
    u = state_from(om, B, lambda X: workloads.isentropic_vortex(X[0], X[1], center=(0.4, 0.6)))
    h = om.cell_widths()
    solver.set_state(u[perm])
    dt = oader.cfl_dt(u, h, P, order, cfl=workloads.ADER_CFL[order])
    solver.compute_dt()
    assert abs(solver.dt.item() - dt) < 1e-13 * dt
    for _ in range(3):
        out = ostep.step(om, u, dt, P, B)
        u, dt = out.u, out.dt_next
    solver.step(3)
    got = solver.get_state().cpu().numpy()
    assert rel_l2(got, u[perm]) < TOL64
    assert abs(solver.dt.item() - dt) < 1e-12 * dt
    assert solver.status() == 0
    assert np.any(solver.skeleton())


def test_remesh_transfer_parity():
    """Refine/coarsen a state-carrying mesh with a moving ball: the library's
    transferred state equals the oracle's (interpolation, L2 projection)."""
    dim, order = 3, 3
    solver, om, perm = build_pair(dim, order, "euler", 3, 2, [(0.5, 0.5, 0.5)] * 2, 0.15)
    B = obasis.Basis(order)
    u = state_from(om, B, lambda X: workloads.density_bubble(X, sigma=0.2))
    solver.set_state(u[perm])
    changed = 0
    for c in [(0.6, 0.55, 0.5), (0.8, 0.7, 0.6), (0.1, 0.9, 0.05)]:
        fl = omesh.sphere_flags(om, c, 0.15)
        before = len(om.cells)
        solver.remesh(fl[perm])
        u = om.remesh(u, fl, B)
        changed += len(om.cells) != before
        keys = lib_keys(solver)
        assert sorted(keys) == om.cells
        perm = np.array([om.index[k] for k in keys])
        assert rel_l2(solver.get_state().cpu().numpy(), u[perm]) < 1e-13
    assert changed >= 2


def test_nonphysical_state_sets_status():
    """A negative density in one cell is reported through the status word
    (the kernels check the state; nothing faults)."""
    solver, om, perm = build_pair(2, 2, "euler", 3, 0)
    B = obasis.Basis(2)
    u = random_state(om, B, "euler", 1)
    u[4, 0] = -1.0
    solver.set_state(u[perm])
    solver.set_dt(1e-3)
    solver.step(1)
    assert solver.status() & 2
    assert solver.status() == 0   # reading clears it


# Tensor-core predictor (tcgen05): stated bounds on every field of one step
# against the FP64 oracle -- 3xTF32 at the FP32 bar (1e-6), 3xBF16 at 5e-6
# (hi + lo carry 16 significant bits); plain TF32 at the bound derived from
# its operand rounding (tf32_operand_tolerance).
TOL_BF16X3 = 5e-6


@pytest.mark.parametrize("order,precision,tol", [
    (5, "tf32x3", TOL32), (5, "bf16x3", TOL_BF16X3), (5, "tf32", None),
    (7, "tf32x3", TOL32), (7, "bf16x3", TOL_BF16X3), (7, "tf32", None), (6, "tf32x3", TOL32),
    (6, "tf32", None)])
def test_tensor_core_predictor_bound(order, precision, tol):
    base, lvl = (3, 1) if order == 5 else (2, 0)
    stage_parity(3, order, "euler", base, lvl, [(0.5, 0.5, 0.5)] * lvl, 0.2, seed=60 + order,
                 tol=tol or 0.0, precision=precision,
                 tol_from=tf32_operand_tolerance if precision == "tf32" else None)


@pytest.mark.parametrize("dim,order,precision,tol", [(2, 3, "fp64", TOL64), (3, 4, "fp64", TOL64),
                                                     (3, 7, "fp64", TOL64), (3, 4, "fp32", TOL32)])
def test_cauchy_kowalevski_predictor(dim, order, precision, tol):
    """Linear acoustics with the Cauchy-Kowalevski predictor on AMR meshes."""
    c = (0.45, 0.5, 0.55)[:dim]
    base, lvl = (9, 2) if dim == 2 else ((3, 2) if order < 7 else (2, 0))
    stage_parity(dim, order, "acoustics", base, lvl, [c] * lvl, 0.12, seed=70 + order, tol=tol,
                 precision=precision, predictor="ck")


def test_solution_based_remesh_parity():
    """Solution-based AMR (first-derivative criterion on the density): the
    device indicator equals the oracle's, flags agree away from the
    thresholds, and a run that remeshes by the criterion every 2 steps keeps
    the same mesh and state as the oracle."""
    from oracle import criterion
    dim, order = 3, 3
    solver, om, perm = build_pair(dim, order, "euler", 5, 2)
    B = obasis.Basis(order)
    P = opde.Euler(dim)
    u = state_from(om, B, lambda X: workloads.density_bubble(X, sigma=0.08))
    solver.set_state(u[perm])
    refine_above, coarsen_below = 0.04, 0.01
    changed = 0
    for rnd in range(3):
        eta_o, fl_o = criterion.gradient_flags(om, u, B, 0, refine_above, coarsen_below)
        eta_g, fl_g = solver.gradient_flags(0, refine_above, coarsen_below)
        assert rel_l2(eta_g, eta_o[perm]) < 1e-12
        eta_a = solver.gradient_indicator(0).cpu().numpy()
        assert np.array_equal(eta_a, eta_g)
        near = (np.abs(eta_o[perm] - refine_above) < 1e-10) | (np.abs(eta_o[perm] - coarsen_below) < 1e-10)
        assert np.array_equal(fl_g[~near], fl_o[perm][~near])
        before = len(om.cells)
        solver.remesh(fl_o[perm])
        u = om.remesh(u, fl_o, B)
        changed += len(om.cells) != before
        keys = lib_keys(solver)
        assert sorted(keys) == om.cells
        perm = np.array([om.index[k] for k in keys])
        h = om.cell_widths()
        dt = oader.cfl_dt(u, h, P, order, cfl=workloads.ADER_CFL[order])
        solver.set_dt(dt)
        for _ in range(2):
            out = ostep.step(om, u, dt, P, B)
            u, dt = out.u, out.dt_next
        solver.step(2)
        assert rel_l2(solver.get_state().cpu().numpy(), u[perm]) < TOL64
    assert changed >= 2
    assert solver.status() == 0


@pytest.mark.parametrize("deriv", [1, 2])
@pytest.mark.parametrize("dim,order,pde,var", [(2, 3, "euler", 0), (2, 7, "euler", 3),
                                               (3, 2, "euler", 4), (3, 5, "euler", 1),
                                               (3, 7, "acoustics", 0), (2, 4, "acoustics", 2)])
def test_gradient_indicator_parity(dim, order, pde, var, deriv):
    """The asynchronous device indicator (first derivatives, or the Hessian)
    on an AMR mesh (a ragged last block of cells in 2D) equals the oracle's
    eta to 1e-12 and the eta returned by gradient_flags bit for bit."""
    from oracle import criterion
    import torch
    base, lvl = (7, 2) if dim == 2 else (3, 1)
    solver, om, perm = build_pair(dim, order, pde, base, lvl, [(0.5, 0.5, 0.5)[:dim]] * lvl)
    B = obasis.Basis(order)
    rng = np.random.default_rng(90 + order)
    if pde == "euler":
        u = workloads.random_euler(rng, dim, (len(om.cells),) + (B.n,) * dim)
    else:
        u = workloads.random_acoustics(rng, dim, (len(om.cells),) + (B.n,) * dim)
    u = np.ascontiguousarray(np.moveaxis(u, 0, 1))
    solver.set_state(u[perm])
    eta_o, fl_o = criterion.gradient_flags(om, u, B, var, 1.0, 0.5, deriv=deriv)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        eta_a = solver.gradient_indicator(var, stream=st, deriv=deriv)
    st.synchronize()
    eta_a = eta_a.cpu().numpy()
    assert rel_l2(eta_a, eta_o[perm]) < 1e-12
    eta_g, fl_g = solver.gradient_flags(var, 1.0, 0.5, deriv=deriv)
    assert np.array_equal(eta_a, eta_g)
    near = (np.abs(eta_o[perm] - 1.0) < 1e-10) | (np.abs(eta_o[perm] - 0.5) < 1e-10)
    assert np.array_equal(fl_g[~near], fl_o[perm][~near])
    from paper_1806_07984_gb300 import ader as A
    with pytest.raises(A.AderError):
        solver.gradient_flags(var, 1.0, 0.5, deriv=3)


# Double-float predictor (pairs of FP32 values, ~48 significant bits): stated
# bound 1e-11 on every field of one step against the FP64 oracle.
TOL_DF64 = 1e-11


@pytest.mark.parametrize("dim,order,pde,base,lvl", [
    (3, 5, "euler", 3, 1), (2, 3, "euler", 9, 2), (3, 3, "euler", 3, 2), (3, 4, "euler", 3, 1),
    (3, 6, "euler", 3, 1), (3, 7, "euler", 3, 1), (2, 7, "euler", 6, 1),
    (3, 5, "acoustics", 3, 1), (2, 4, "acoustics", 9, 1)])
def test_double_float_predictor_bound(dim, order, pde, base, lvl):
    c = (0.5, 0.5, 0.5)[:dim]
    stage_parity(dim, order, pde, base, lvl, [c] * lvl, 0.2, seed=80 + order, tol=TOL_DF64,
                 precision="df64")
