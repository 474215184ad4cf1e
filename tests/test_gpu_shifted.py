"""Global time stepping with a prescribed dt by the shifted task graph (Sec. 3:
when the admissible time step sizes are known, the pass that finishes step k
also runs the predictor of step k + 1): ader_step_fixed_dt runs the corrector
of step k as a prologue of the predictor kernel of step k + 1.

Its state must equal nsteps rounds of ader_predict, ader_riemann and
ader_correct with the same dt bit for bit (the same arithmetic in the same
order, only in one kernel), in every predictor variant, and (FP64) the
oracle's nsteps steps with that dt; the CFL time step of the final state must
equal the staged corrector's."""
import numpy as np
import pytest

from oracle import ader as oader, basis as obasis, pde as opde, step as ostep
import workloads
from gpu_helpers import build_pair, close_fields
from oracle_helpers import random_state

pytestmark = pytest.mark.gpu

CASES = [
    # dim, order, pde, base, levels, precision, predictor
    (2, 3, "euler", 9, 2, "fp64", "picard"),
    (3, 3, "euler", 3, 1, "fp64", "picard"),
    (3, 5, "euler", 3, 1, "fp64", "picard"),
    (3, 5, "euler", 3, 1, "fp32", "picard"),
    (3, 5, "euler", 3, 1, "df64", "picard"),
    (3, 5, "euler", 3, 1, "tf32x3", "picard"),
    (3, 4, "acoustics", 3, 1, "fp64", "ck"),
    (2, 5, "acoustics", 9, 1, "fp64", "picard"),
]


def _pair(dim, order, pde, base, levels, precision, predictor, seed):
    centers = [(0.4, 0.55, 0.5)[:dim]] * levels
    made = []
    for _ in range(2):
        s, om, perm = build_pair(dim, order, pde, base, levels, centers, 0.2,
                                 precision=precision, predictor=predictor)
        made.append(s)
    B = obasis.Basis(order)
    u0 = random_state(om, B, pde, seed)
    return made, om, perm, B, u0


@pytest.mark.parametrize("dim,order,pde,base,levels,precision,predictor", CASES)
def test_shifted_steps_equal_staged_steps(dim, order, pde, base, levels, precision, predictor):
    import torch
    (staged, shifted), om, perm, B, u0 = _pair(dim, order, pde, base, levels, precision, predictor,
                                               seed=70 + 7 * dim + order)
    P = opde.make_pde(pde, dim)
    dt = 0.5 * oader.cfl_dt(u0, om.cell_widths(), P, order, cfl=workloads.ADER_CFL[order])
    nsteps = 4
    for s in (staged, shifted):
        s.set_state(u0[perm])
        s.set_dt(dt)
    dt_a = torch.zeros(1, dtype=torch.float64, device=staged.device)
    for _ in range(nsteps):
        staged.predict()
        staged.riemann()
        staged.correct(dt_a)           # dt_a receives the CFL step; staged.dt stays dt
    dt_b = torch.zeros(1, dtype=torch.float64, device=shifted.device)
    shifted.step_fixed_dt(nsteps, dt_b)
    ua = staged.get_state().cpu().numpy()
    ub = shifted.get_state().cpu().numpy()
    assert np.array_equal(ua, ub), np.abs(ua - ub).max()
    assert dt_a.item() == dt_b.item() and dt_b.item() > 0
    assert shifted.dt.item() == dt               # the prescribed dt is read only
    assert staged.status() == 0 and shifted.status() == 0
    if precision == "fp64":
        u = u0
        for _ in range(nsteps):
            ref = ostep.step(om, u, dt, P, B, predictor=predictor)
            u = ref.u
        assert close_fields(ub, u[perm], 1e-12)
        assert abs(dt_b.item() - ref.dt_next) < 1e-12 * ref.dt_next
    for s in (staged, shifted):
        s.close()


def test_shifted_zero_and_one_step():
    import torch
    (staged, shifted), om, perm, B, u0 = _pair(3, 3, "euler", 3, 1, "fp64", "picard", seed=91)
    P = opde.Euler(3)
    dt = 0.5 * oader.cfl_dt(u0, om.cell_widths(), P, 3, cfl=workloads.ADER_CFL[3])
    for s in (staged, shifted):
        s.set_state(u0[perm])
        s.set_dt(dt)
    shifted.step_fixed_dt(0)
    assert np.array_equal(shifted.get_state().cpu().numpy(), u0[perm])
    dt_a = torch.zeros(1, dtype=torch.float64, device=staged.device)
    staged.predict()
    staged.riemann()
    staged.correct(dt_a)
    shifted.step_fixed_dt(1)                      # dt_next discarded
    assert np.array_equal(staged.get_state().cpu().numpy(), shifted.get_state().cpu().numpy())
    for s in (staged, shifted):
        s.close()


def test_shifted_steps_reject_limiter_and_negative_counts():
    from paper_1806_07984_gb300 import ader as A
    s, om, perm = build_pair(2, 3, "euler", 9, 0, limiter=True)
    B = obasis.Basis(3)
    s.set_state(random_state(om, B, "euler", 5)[perm])
    s.set_dt(1e-4)
    with pytest.raises(A.AderError):
        s.step_fixed_dt(2)
    s.close()
    s, om, perm = build_pair(2, 3, "euler", 9, 0)
    with pytest.raises(A.AderError):
        s.step_fixed_dt(-1)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_shifted_steps_full_size(precision):
    """The 3D N=5 bench mesh (base 27^3, two levels around the bubble,
    268,087 cells): two shifted steps equal two staged steps bit for bit."""
    import torch
    from paper_1806_07984_gb300 import Solver
    runs = []
    for shifted in (False, True):
        s = Solver(3, 5, "euler", base=(27, 27, 27), max_level=2, cfl=workloads.ADER_CFL[5],
                   precision=precision)
        center = workloads.sphere_center(0.0)
        for _ in range(2):
            s.remesh(s.sphere_flags(center, 0.15))
        s.classify(s.sphere_flags(center, 0.15))
        assert s.ncells == 268087
        X = s.node_coords()
        s.set_state(torch.from_numpy(np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X), 0, 1))).cuda())
        del X
        s.compute_dt()
        dt_next = torch.zeros(1, dtype=torch.float64, device=s.device)
        if shifted:
            s.step_fixed_dt(2, dt_next)
        else:
            for _ in range(2):
                s.predict()
                s.riemann()
                s.correct(dt_next)
        runs.append((s.get_state().cpu().numpy(), dt_next.item(), s.status()))
        s.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1] and runs[0][2] == runs[1][2] == 0
