"""Parity at the bench's full sizes: 3D Euler on base 27^3 with two levels
around the bubble (268,087 cells) at N=5 (the FP64 headline workload) and at
N=7 (the mixed-precision workload: FP64, double-float, FP32 and the tcgen05
3xTF32 / 3xBF16 predictors), in the launch configuration the bench times
(ader_step on the two prioritised streams, enclave pipeline).  The oracle
cannot run the whole mesh in seconds, so it evaluates sampled cells one by
one (step_sample) on its own independently built mesh; a conservation
property is checked on all cells."""
import numpy as np
import pytest

from oracle import ader as oader, basis as obasis, mesh as omesh, pde as opde, step as ostep
import workloads
from gpu_helpers import lib_keys, rel_l2, rel_max

pytestmark = pytest.mark.gpu

DIM, BASE, LEVELS, RADIUS = 3, 27, 2, 0.15
# Tensor-core split predictors: 3xTF32 at the FP32 bar, 3xBF16 at 5e-6 (hi +
# lo BF16 parts carry 16 significant bits).
TOL_BF16X3 = 5e-6

_PROBLEMS = {}


def full_problem(order):
    """Oracle mesh and initial state at order N (kept for the module)."""
    if order in _PROBLEMS:
        return _PROBLEMS[order]
    _PROBLEMS.clear()                      # one order's state in host memory at a time
    B = obasis.Basis(order)
    om = omesh.Mesh(DIM, (BASE,) * DIM, LEVELS)
    center = workloads.sphere_center(0.0)
    flag_seq = []
    for _ in range(LEVELS):
        fl = omesh.sphere_flags(om, center, RADIUS)
        flag_seq.append(fl)
        om.remesh(np.zeros((len(om.cells), 1, 2, 2, 2)), fl, obasis.Basis(1))
    X = om.node_coords(B.xi)
    u = np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X), 0, 1))
    del X
    _PROBLEMS[order] = (om, B, u)
    return om, B, u


def lib_solver(precision, om, order):
    from paper_1806_07984_gb300 import Solver
    s = Solver(DIM, order, "euler", base=(BASE,) * 3, max_level=LEVELS,
               cfl=workloads.ADER_CFL[order], precision=precision)
    center = workloads.sphere_center(0.0)
    ref = omesh.Mesh(DIM, (BASE,) * DIM, LEVELS)
    for _ in range(LEVELS):
        fl = s.sphere_flags(center, RADIUS)
        fo = omesh.sphere_flags(ref, center, RADIUS)
        perm = [ref.index[k] for k in lib_keys(s)]
        assert np.array_equal(fl, fo[perm])          # host criterion agrees
        s.remesh(fl)
        ref.remesh(np.zeros((len(ref.cells), 1, 2, 2, 2)), fo, obasis.Basis(1))
    s.classify(s.sphere_flags(center, RADIUS))
    keys = lib_keys(s)
    assert sorted(keys) == om.cells                  # same adaptive mesh
    return s, np.array([om.index[k] for k in keys])


def integrals(u, h, B):
    y = u
    for _ in range(DIM):
        y = np.tensordot(y, B.w, axes=([y.ndim - 1], [0]))
    return (y * np.prod(h, axis=1)[:, None]).sum(axis=0)


@pytest.mark.parametrize("order,precision,tol", [
    (5, "fp64", 1e-12), (5, "df64", 1e-11), (5, "fp32", 1e-6),
    (7, "fp64", 1e-12), (7, "df64", 1e-11), (7, "fp32", 1e-6), (7, "tf32x3", 1e-6),
    (7, "bf16x3", TOL_BF16X3)])
def test_full_size_sampled_parity(order, precision, tol):
    om, B, u = full_problem(order)
    P = opde.Euler(DIM)
    h = om.cell_widths()
    dt = oader.cfl_dt(u, h, P, order, cfl=workloads.ADER_CFL[order])
    s, perm = lib_solver(precision, om, order)
    assert s.ncells == len(om.cells) == 268087
    s.set_state(u[perm])
    s.set_dt(dt)
    s.step(1)
    got = s.get_state().cpu().numpy()
    assert s.status() == 0
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    # sampled cells: skeleton (both sides of transitions), enclave, first/last
    rng = np.random.default_rng(5)
    skel = np.flatnonzero(s.skeleton())
    encl = np.flatnonzero(~s.skeleton().astype(bool))
    lib_t = np.concatenate([rng.choice(skel, 12, replace=False), rng.choice(encl, 12, replace=False),
                            [0, s.ncells - 1]])
    or_t = perm[lib_t]
    ref = ostep.step_sample(om, u, dt, P, B, or_t)
    for a, b in zip(got[lib_t], ref):
        assert rel_l2(a, b) < tol
        assert rel_max(a, b) <= 10 * tol
    if precision in ("fp64", "df64"):
        # the increment u(T+dt) - u(T) itself, not only the state
        assert rel_l2(got[lib_t] - u[or_t], ref - u[or_t]) < (1e-9 if precision == "fp64" else 1e-8)
    # conservation over the whole mesh (periodic domain, hanging faces)
    I0 = integrals(u, h, B)
    I1 = integrals(got, h[perm], B)
    assert np.allclose(I1, I0, rtol=0, atol=1e-11), I1 - I0
    s.close()
