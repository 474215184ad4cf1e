"""Domain decomposition on one GPU: several sub-domains of one adaptive mesh
in one process (virtual ranks, device copies between their exchange
buffers) against the unpartitioned context, bit for bit, over several steps
and a remesh whose rebalanced cuts move cells between ranks."""
import numpy as np
import pytest

import workloads
from paper_1806_07984_gb300 import ader as A

pytestmark = pytest.mark.gpu


def _pair(dim, order, base, levels, center, radius, nranks, sigma=0.1, pde="euler",
          precision="fp64", predictor="picard"):
    from paper_1806_07984_gb300 import Solver
    from paper_1806_07984_gb300.domain import LocalExchange, SubDomain

    def make():
        s = Solver(dim, order, pde, base=(base,) * 3, max_level=levels,
                   cfl=workloads.ADER_CFL[order], precision=precision, predictor=predictor)
        for _ in range(levels):
            s.remesh(s.sphere_flags(center, radius))
        return s

    ref = make()
    X = ref.node_coords()
    q = workloads.density_bubble(X, sigma=sigma, center=(0.5, 0.5, 0.5)[:dim],
                                 vel=(1.0, 1.0, 1.0)[:dim]) if pde == "euler" else \
        workloads.acoustic_pulses(X, seed=4, width=0.1)
    u = np.ascontiguousarray(np.moveaxis(q, 0, 1))
    ref.set_state(u)
    ref.compute_dt()
    subs = []
    for r in range(nranks):
        s = make()
        s.set_state(u)
        s.dt.copy_(ref.dt)
        subs.append(SubDomain(s, nranks, r))
    return ref, subs, LocalExchange(subs)


def _gather(subs):
    import torch
    return torch.cat([s.solver.get_state().reshape(-1) for s in subs])


@pytest.mark.parametrize("dim,order,base,levels,nranks,pde,precision,predictor", [
    (2, 3, 9, 2, 3, "euler", "fp64", "picard"), (3, 3, 5, 1, 4, "euler", "fp64", "picard"),
    (2, 5, 9, 2, 2, "euler", "fp64", "picard"), (3, 5, 5, 1, 3, "euler", "fp32", "picard"),
    (2, 4, 9, 2, 3, "euler", "df64", "picard"), (3, 4, 5, 1, 3, "acoustics", "fp64", "ck")])
def test_subdomains_equal_whole_mesh_bitwise(dim, order, base, levels, nranks, pde, precision,
                                             predictor):
    from paper_1806_07984_gb300.domain import remesh_local, step_local
    center = (0.45, 0.5, 0.55)[:dim]
    ref, subs, ex = _pair(dim, order, base, levels, center, 0.2, nranks, pde=pde,
                          precision=precision, predictor=predictor)
    info = [s.info() for s in subs]
    assert sum(i[4] for i in info) == ref.ncells
    assert all(i[5] > 0 for i in info)                     # every rank has ghosts
    assert sum(s.halo_bytes() for s in subs) > 0
    cuts0 = subs[0].cuts()
    for rnd in range(2):
        ref.step(3)
        step_local(subs, ex, 3)
        got = _gather(subs)
        assert got.numel() == ref.get_state().numel()
        assert bool((got == ref.get_state().reshape(-1)).all()), rnd
        assert float(subs[0].solver.dt.item()) == float(ref.dt.item())
        # move the refined ball: every rank adapts with the same whole-mesh flags
        c = tuple(x + 0.12 * (rnd + 1) for x in center)
        flags = ref.sphere_flags(c, 0.2)
        for s in subs:
            assert np.array_equal(s.solver.sphere_flags(c, 0.2), flags)
        ref.remesh(flags)
        remesh_local(subs, ex, flags)
        got = _gather(subs)
        assert bool((got == ref.get_state().reshape(-1)).all()), ("after remesh", rnd)
    assert not np.array_equal(subs[0].cuts(), cuts0)          # the cuts were rebalanced
    ref.step(2)
    step_local(subs, ex, 2)
    assert bool((_gather(subs) == ref.get_state().reshape(-1)).all())
    assert ref.status() == 0 and all(s.solver.status() == 0 for s in subs)
    for s in subs:
        s.solver.close()
    ref.close()


def test_partitioned_context_rejects_whole_mesh_calls():
    from paper_1806_07984_gb300 import Solver
    from paper_1806_07984_gb300.domain import SubDomain
    s = Solver(2, 2, "euler", base=(6, 6, 1), max_level=0, cfl=workloads.ADER_CFL[2])
    sub = SubDomain(s, 2, 1)
    with pytest.raises(A.AderError):
        s.step(1)
    with pytest.raises(A.AderError):
        A.ader_partition(s.ctx, 2, 0)
    with pytest.raises(A.AderError):
        A.ader_halo_size(s.ctx, 2)
    assert sub.info()[:2] == (2, 1) and sub.info()[2] == 36
    s.close()
