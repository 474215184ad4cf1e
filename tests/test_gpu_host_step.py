"""ader_step_host: one step with the state copied in from and out to host
memory, the copy in overlapped with the enclave predictor chunks, equals
set_state + ader_step + get_state bit for bit (AMR mesh, several steps, a
remesh in between, pipelined and plain steps)."""
import numpy as np
import pytest

import workloads
from paper_1806_07984_gb300 import ader as A

pytestmark = pytest.mark.gpu


def _pair(chunks):
    from paper_1806_07984_gb300 import Solver
    out = []
    for _ in range(2):
        s = Solver(3, 3, "euler", base=(9, 9, 9), max_level=2, cfl=workloads.ADER_CFL[3],
                   pipeline_chunks=chunks)
        for _ in range(2):
            s.remesh(s.sphere_flags((0.5, 0.5, 0.5), 0.15))
        s.classify(s.sphere_flags((0.5, 0.5, 0.5), 0.15))
        out.append(s)
    return out


@pytest.mark.parametrize("chunks", [8, 1])
def test_host_step_equals_device_step(chunks):
    import torch
    ref, s = _pair(chunks)
    X = ref.node_coords()
    u = np.ascontiguousarray(np.moveaxis(workloads.density_bubble(X, sigma=0.08), 0, 1))
    ref.set_state(u)
    ref.compute_dt()
    s.set_state(u)
    s.compute_dt()
    host = torch.from_numpy(u.copy()).pin_memory()
    for rnd in range(2):
        for _ in range(3):
            ref.step(1)
            A.ader_step_host(s.ctx, host.data_ptr(), host.data_ptr(), s.dt.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(host.numpy(), ref.get_state().cpu().numpy()), rnd
        assert s.dt.item() == ref.dt.item()
        if rnd == 0:
            fl = ref.sphere_flags((0.62, 0.55, 0.5), 0.15)
            ref.remesh(fl)
            s.set_state(host.numpy())
            s.remesh(fl)
            host = s.get_state().cpu().pin_memory()
    assert ref.status() == 0 and s.status() == 0
    ref.close()
    s.close()
