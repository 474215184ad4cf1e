"""GPU parity of the a posteriori subcell FV limiter against the oracle:
forced limiting (all cells, a seeded subset, at a resolution transition),
detection on a circular explosion over several steps, flags, conservation
and the next time step."""
import numpy as np
import pytest

from oracle import ader as oader, basis as obasis, limiter as olim, pde as opde
from gpu_helpers import build_pair, rel_l2
from oracle_helpers import random_state
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-12


def flags_of(out):
    f = np.zeros(len(out.limited), dtype=np.uint32)
    f |= out.limited.astype(np.uint32)
    f |= 2 * out.fixed.astype(np.uint32)
    f |= 4 * out.kept.astype(np.uint32)
    return f


def limited_step_parity(solver, om, perm, u0, P, B, force=None, steps=1):
    """Run `steps` limited steps on both sides; compare state, flags, dt."""
    h = om.cell_widths()
    dt = oader.cfl_dt(u0, h, P, B.order)
    u = u0
    solver.set_state(u0[perm])
    solver.set_dt(dt)
    if force is not None:
        solver.force_limit(force[perm])
    outs = []
    for _ in range(steps):
        ref = olim.step_limited(om, u, dt, P, B, force=force)
        solver.step(1)
        got = solver.get_state().cpu().numpy()
        flags, nlim = solver.limiter_flags()
        assert np.array_equal(flags, flags_of(ref)[perm])
        assert nlim == int(ref.limited.sum())
        assert rel_l2(got, ref.u[perm]) < TOL
        assert rel_l2(got - u[perm], ref.u[perm] - u[perm]) < 1e-9
        assert abs(solver.dt.item() - ref.dt_next) < TOL * ref.dt_next
        outs.append(ref)
        u, dt = ref.u, ref.dt_next
    return outs


@pytest.mark.parametrize("dim,order,base", [(2, 3, 4), (2, 7, 3), (3, 2, 3), (3, 5, 3), (3, 7, 3)])
def test_all_cells_limited(dim, order, base):
    solver, om, perm = build_pair(dim, order, "euler", base, 0, limiter=True)
    B = obasis.Basis(order)
    P = opde.make_pde("euler", dim)
    u0 = random_state(om, B, "euler", seed=40 + order)
    force = np.ones(len(om.cells), dtype=bool)
    limited_step_parity(solver, om, perm, u0, P, B, force)
    assert solver.status() == 0


@pytest.mark.parametrize("dim,order,base,pde", [(2, 3, 6, "euler"), (3, 3, 3, "euler"),
                                                (3, 5, 3, "euler"), (3, 6, 3, "euler"),
                                                (2, 4, 5, "acoustics"), (3, 2, 3, "acoustics"),
                                                (3, 7, 3, "acoustics")])
def test_forced_subset_conserves(dim, order, base, pde):
    solver, om, perm = build_pair(dim, order, pde, base, 0, limiter=True)
    B = obasis.Basis(order)
    P = opde.make_pde(pde, dim)
    u0 = random_state(om, B, pde, seed=50 + order)
    force = np.random.default_rng(order).random(len(om.cells)) < 0.3
    outs = limited_step_parity(solver, om, perm, u0, P, B, force, steps=2)
    assert outs[0].fixed.any()
    h = om.cell_widths()
    inv = np.argsort(perm)
    got = solver.get_state().cpu().numpy()[inv]
    I0 = oader.cell_integral(u0, h, B)
    assert np.allclose(oader.cell_integral(got, h, B), I0, atol=1e-12, rtol=0)


def test_transition_cells_keep_dg():
    solver, om, perm = build_pair(2, 3, "euler", 9, 1, centers=[(0.5, 0.5)], radius=0.1,
                                  limiter=True)
    B = obasis.Basis(3)
    P = opde.Euler(2)
    u0 = random_state(om, B, "euler", seed=7)
    nb = olim.neighbors(om)
    at_tr = ~(nb >= 0).all(axis=(1, 2))
    force = np.zeros(len(om.cells), dtype=bool)
    force[np.flatnonzero(at_tr)[:3]] = True
    force[np.flatnonzero(~at_tr)[::7]] = True
    outs = limited_step_parity(solver, om, perm, u0, P, B, force)
    assert outs[0].kept[force & at_tr].all() and outs[0].limited[force & ~at_tr].all()
    assert solver.status() == 32          # reported, and the step is otherwise clean


@pytest.mark.parametrize("dim,order,base,steps", [(2, 3, 27, 3), (3, 2, 9, 1)])
def test_explosion_detection(dim, order, base, steps):
    solver, om, perm = build_pair(dim, order, "euler", base, 0, limiter=True)
    B = obasis.Basis(order)
    P = opde.Euler(dim)
    X = om.node_coords(B.xi)
    u0 = np.ascontiguousarray(np.moveaxis(workloads.circular_explosion(X, width=0.02), 0, 1))
    outs = limited_step_parity(solver, om, perm, u0, P, B, steps=steps)
    assert all(0 < o.limited.sum() < len(om.cells) // 2 for o in outs)
    assert solver.status() == 0


def test_limiter_off_by_default():
    from paper_1806_07984_gb300 import Solver, ader as A
    s = Solver(2, 3, "euler", base=(3, 3, 1), cfl=workloads.ADER_CFL[3])
    with pytest.raises(A.AderError):
        s.limiter_flags()
    with pytest.raises(A.AderError):
        s.force_limit(np.ones(9, dtype=bool))


def test_pipeline_chunks_do_not_change_the_result():
    """ader_step with the enclave predictor in K chunks (faces and correctors
    overlapping later chunks) equals the unchunked step bit for bit, on an AMR
    mesh with remeshing and with the limiter."""
    from paper_1806_07984_gb300 import Solver
    import torch
    results = []
    for K, lim, ctas in ((1, False, 0), (3, False, 2), (8, False, 1), (1, True, 0), (5, True, 3)):
        s = Solver(3, 3, "euler", base=(9, 9, 9), max_level=1, cfl=workloads.ADER_CFL[3],
                   pipeline_chunks=K, limiter=lim, pipeline_ctas=ctas)
        s.remesh(s.sphere_flags((0.5, 0.5, 0.5), 0.2))
        s.classify(s.sphere_flags((0.5, 0.5, 0.5), 0.2))
        X = s.node_coords()
        u0 = np.ascontiguousarray(np.moveaxis(
            workloads.circular_explosion(X, width=0.5 / 9), 0, 1))
        s.set_state(torch.from_numpy(u0).cuda())
        s.compute_dt()
        s.step(2)
        s.remesh(s.sphere_flags((0.55, 0.5, 0.5), 0.2))
        s.step(2)
        results.append((s.get_state().cpu().numpy(), s.dt.item(), s.status()))
        s.close()
    for r in results[1:3]:
        assert np.array_equal(r[0], results[0][0]) and r[1] == results[0][1]
    assert np.array_equal(results[4][0], results[3][0]) and results[4][1] == results[3][1]
    assert not np.array_equal(results[3][0], results[0][0])   # the limiter acted


def test_refinement_follows_the_shock():
    """Limited steps with a remesh after each that refines around the
    troubled cells (and coarsens elsewhere): flags, meshes and states equal
    the oracle's."""
    from gpu_helpers import lib_keys
    solver, om, perm = build_pair(2, 3, "euler", 27, 1, limiter=True)
    B = obasis.Basis(3)
    P = opde.Euler(2)
    X = om.node_coords(B.xi)
    u = np.ascontiguousarray(np.moveaxis(workloads.circular_explosion(X, width=0.02), 0, 1))
    solver.set_state(u[perm])
    for cycle in range(3):
        h = om.cell_widths()
        dt = oader.cfl_dt(u, h, P, 3)
        solver.compute_dt()
        assert abs(solver.dt.item() - dt) < TOL * dt
        ref = olim.step_limited(om, u, dt, P, B)
        solver.step(1)
        assert rel_l2(solver.get_state().cpu().numpy(), ref.u[perm]) < TOL
        fl_ref = olim.refine_flags(om, ref.limited | ref.kept)
        fl_gpu = solver.limiter_refine_flags()
        assert np.array_equal(fl_gpu, fl_ref[perm])
        troubled = ref.limited | ref.kept
        assert troubled.any() and (fl_ref[troubled] >= 0).all()
        if cycle == 0:
            assert (fl_ref > 0).any()
        u = om.remesh(ref.u, fl_ref, B)
        solver.remesh(fl_gpu)
        keys = lib_keys(solver)
        assert sorted(keys) == om.cells
        perm = np.array([om.index[k] for k in keys])
        assert rel_l2(solver.get_state().cpu().numpy(), u[perm]) < TOL
    assert max(k[0] for k in om.cells) == 1


def test_troubled_transition_cells_refine_and_redo():
    """ader_step_refining: an explosion front crossing the transitions of a
    refined patch; while troubled cells sit at a transition the step goes
    back to u(T), refines around the troubled cells (refinement only) and
    runs again.  The oracle takes the same steps (its limiter, its refine
    flags without the coarsening, its transfer): rounds, meshes, flags and
    states agree, and no troubled cell is left at a transition."""
    from gpu_helpers import lib_keys
    solver, om, perm = build_pair(2, 3, "euler", 27, 2, centers=[(0.5, 0.75)], radius=0.06,
                                  limiter=True)
    B = obasis.Basis(3)
    P = opde.Euler(2)
    X = om.node_coords(B.xi)
    u = np.ascontiguousarray(np.moveaxis(workloads.circular_explosion(X, width=0.02), 0, 1))
    solver.set_state(u[perm])
    solver.compute_dt()
    all_rounds = []
    dt = oader.cfl_dt(u, om.cell_widths(), P, 3)
    for cycle in range(2):
        r = 0
        while True:
            ref = olim.step_limited(om, u, dt, P, B)
            if not ref.kept.any() or r == 3:
                break
            fl = np.maximum(olim.refine_flags(om, ref.limited | ref.kept), 0).astype(np.int8)
            u = om.remesh(u, fl, B)
            dt = oader.cfl_dt(u, om.cell_widths(), P, 3)
            r += 1
        got_r = solver.step_refining(max_rounds=3)
        assert got_r == r, (cycle, got_r, r)
        all_rounds.append(r)
        keys = lib_keys(solver)
        assert sorted(keys) == om.cells
        perm = np.array([om.index[k] for k in keys])
        flags, nlim = solver.limiter_flags()
        assert np.array_equal(flags, flags_of(ref)[perm])
        assert rel_l2(solver.get_state().cpu().numpy(), ref.u[perm]) < TOL
        assert abs(solver.dt.item() - ref.dt_next) < TOL * ref.dt_next
        assert not ref.kept.any()
        assert solver.status() == 0       # the discarded attempts' bits are dropped
        u, dt = ref.u, ref.dt_next       # dt_next includes the limited cells' subcells
    assert all_rounds[0] >= 2 and all_rounds[1] == 0
    with pytest.raises(Exception):
        from paper_1806_07984_gb300 import Solver
        plain = Solver(2, 2, "euler", base=(3, 3, 1), cfl=0.1)
        try:
            plain.step_refining()
        finally:
            plain.close()


def test_default_chunks_follow_the_mesh_size():
    """pipeline_chunks = 0 keeps the pipeline off on a small mesh (729 cells:
    fewer launches per step than 8 explicit chunks, the same state bit for
    bit) and turns it on when remeshing makes the enclave large enough (the
    27^2 base refined everywhere twice: 59,049 cells, 3,691 predictor CTAs of
    16 cells, 8 CTAs per SM per chunk)."""
    from paper_1806_07984_gb300 import Solver
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_step, states = {}, {}
    for K in (0, 8, 1):
        s = Solver(2, 3, "euler", base=(27, 27, 1), max_level=2, cfl=workloads.ADER_CFL[3],
                   pipeline_chunks=K, eager_steps=True)
        X = s.node_coords()
        u0 = np.ascontiguousarray(np.moveaxis(workloads.isentropic_vortex(X[0], X[1]), 0, 1))
        s.set_state(torch.from_numpy(u0).cuda())
        s.compute_dt()
        n0 = s.launch_count()
        s.step(2)
        per_step[K] = (s.launch_count() - n0) / 2
        states[K] = (s.get_state().cpu().numpy(), s.dt.item())
        if K == 0:
            for _ in range(2):
                s.remesh(np.ones(s.ncells, dtype=np.int8))
            assert s.ncells == 59049
            n0 = s.launch_count()
            s.step(1)
            big = s.launch_count() - n0
            assert s.status() == 0
        s.close()
    assert per_step[0] == per_step[1] < per_step[8]
    assert np.array_equal(states[0][0], states[8][0]) and states[0][1] == states[8][1]
    assert np.array_equal(states[0][0], states[1][0])
    k_big = max(1, min(8, ((59049 + 15) // 16) // (8 * sms)))
    assert (big > per_step[1]) == (k_big > 1)
