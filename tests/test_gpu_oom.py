"""Buffer growth under allocation failure, injected on the host: every
allocation point of a growing remesh fails in turn; each failure returns
ADER_ERR_OOM and leaves mesh and state as before the call, and the context
then remeshes and steps exactly like one that never failed."""
import numpy as np
import pytest

import workloads
from paper_1806_07984_gb300 import ader as A

pytestmark = pytest.mark.gpu


def _solver():
    from paper_1806_07984_gb300 import Solver
    s = Solver(3, 3, "euler", base=(5, 5, 5), max_level=2, cfl=workloads.ADER_CFL[3])
    X = s.node_coords()
    s.set_state(np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X, sigma=0.1), 0, 1)))
    s.compute_dt()
    return s


def test_remesh_survives_allocation_failures():
    ref, s = _solver(), _solver()
    flags = ref.sphere_flags((0.5, 0.5, 0.5), 0.25)
    u0, cells0 = s.get_state().clone(), s.cells().copy()
    failures = 0
    try:
        for k in range(64):
            A.ader_debug_fail_allocations(k)
            try:
                s.remesh(flags)
            except A.AderError as e:
                A.ader_debug_fail_allocations(-1)
                assert e.status == -3, e
                failures += 1
                assert np.array_equal(s.cells(), cells0)
                assert bool((s.get_state() == u0).all())
                continue
            break
    finally:
        A.ader_debug_fail_allocations(-1)
    assert failures >= 3          # the cell buffers, the old state's copy and the lists
    ref.remesh(flags)
    assert s.ncells > len(cells0)
    assert np.array_equal(s.cells(), ref.cells())
    assert bool((s.get_state() == ref.get_state()).all())
    for _ in range(2):
        s.step(1)
        ref.step(1)
    assert bool((s.get_state() == ref.get_state()).all())
    assert s.status() == 0 and ref.status() == 0
    s.close()
    ref.close()
