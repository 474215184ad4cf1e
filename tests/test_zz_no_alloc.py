"""The allocation-free time step, ader_compute_dt_static, against the
context's ader_compute_dt.

ader_compute_dt_static exists for callers that cannot allocate device memory
(code inside a memory pool or arena it does not own, or a path that must not
fail for lack of memory): it keeps its scratch in a fixed device array inside
the library.  This file is collected last on purpose; it must pass both on
its own in a fresh process and after every other test.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _levels(solver, torch):
    lv = solver.cells()[:, 0].astype(np.int8)
    return torch.from_numpy(lv).to(solver.device)


def _static_dt(A, solver, u_dev, lv_dev, torch):
    cfg = solver.cfg
    dt = torch.full((1,), -1.0, dtype=torch.float64, device=solver.device)
    A.ader_compute_dt_static(cfg.dim, cfg.order, cfg.pde, cfg.gamma, cfg.cfl,
                             list(cfg.base), list(cfg.lo), list(cfg.hi), solver.ncells,
                             u_dev.data_ptr(), lv_dev.data_ptr(), dt.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return dt.item()


# 3D N=3: 256-thread CTAs; 2D N=5: 252 and 3D N=5: 216 threads, whose last
# warp is partial; 3D N=7: one cell of 512 nodes per CTA.
@pytest.mark.parametrize("dim,order", [(3, 3), (2, 5), (3, 5), (3, 7)])
def test_static_dt_matches_context_dt_twice(dim, order):
    import torch
    from paper_1806_07984_gb300 import Solver, ader as A
    s = Solver(dim, order, "euler", base=(5, 5, 5) if dim == 3 else (9, 9, 1), max_level=1,
               cfl=workloads.ADER_CFL[order])
    center = (0.5, 0.5, 0.5)[:dim]
    s.remesh(s.sphere_flags(center, 0.2))
    X = s.node_coords()
    u = np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X, sigma=0.1), 0, 1))
    s.set_state(u)
    lv = _levels(s, torch)
    results = []
    for call in range(2):
        ref = s.compute_dt().item()
        got = _static_dt(A, s, s.get_state(), lv, torch)
        assert abs(got - ref) <= TOL * ref, (call, got, ref)
        results.append(got)
        s.step(1)              # new state for the second call
    assert s.status() == 0
    s.close()


def test_static_dt_rejects_too_many_cells():
    import torch
    from paper_1806_07984_gb300 import ader as A
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    lv = torch.zeros(1, dtype=torch.int8, device="cuda")
    with pytest.raises(A.AderError) as e:
        A.ader_compute_dt_static(3, 3, A.ADER_EULER, 1.4, 0.1, [3, 3, 3], [0, 0, 0], [1, 1, 1],
                                 A.ADER_DT_STATIC_MAX_CELLS + 1, dummy.data_ptr(), lv.data_ptr(),
                                 dummy.data_ptr())
    assert e.value.status == -1


def _bubble_solver(dim, order):
    from paper_1806_07984_gb300 import Solver
    s = Solver(dim, order, "euler", base=(5, 5, 5) if dim == 3 else (9, 9, 1), max_level=1,
               cfl=workloads.ADER_CFL[order])
    s.remesh(s.sphere_flags((0.5, 0.5, 0.5)[:dim], 0.2))
    X = s.node_coords()
    u = np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X, sigma=0.1), 0, 1))
    s.set_state(u)
    return s, u


@pytest.mark.parametrize("dim,order", [(3, 5), (2, 5)])
def test_static_dt_is_nan_for_negative_pressure(dim, order):
    import torch
    from paper_1806_07984_gb300 import ader as A
    s, u = _bubble_solver(dim, order)
    bad = u.copy()
    flat = bad.reshape(bad.shape[0], bad.shape[1], -1)
    flat[s.ncells // 2, dim + 1, 3] = -1.0       # E < kinetic energy: p < 0
    u_dev = torch.from_numpy(bad).to(s.device)
    assert np.isnan(_static_dt(A, s, u_dev, _levels(s, torch), torch))
    # the same call on the good state is finite again (nothing sticks)
    got = _static_dt(A, s, torch.from_numpy(u).to(s.device), _levels(s, torch), torch)
    assert abs(got - s.compute_dt().item()) <= TOL * got
    s.close()


def test_static_dt_is_nan_for_level_out_of_range():
    import torch
    from paper_1806_07984_gb300 import ader as A
    s, _ = _bubble_solver(3, 3)
    lv = _levels(s, torch)
    lv[s.ncells // 3] = 8
    assert np.isnan(_static_dt(A, s, s.get_state(), lv, torch))
    lv[s.ncells // 3] = -1
    assert np.isnan(_static_dt(A, s, s.get_state(), lv, torch))
    s.close()
