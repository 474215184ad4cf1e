"""Convenience wrapper over the C ABI: one ADER-DG context with torch
device buffers for dt and the state, and torch streams."""
import numpy as np

from . import ader as A


class Solver:
    """An ADER-DG problem on the device.

    State arrays use the library layout u[c][var][node] (node index with x
    fastest), which as a numpy/torch array of shape (C, m, n_z, n_y, n_x)
    (3D) or (C, m, n_y, n_x) (2D) is a C-contiguous view of the same memory.
    """

    def __init__(self, dim, order, pde="euler", base=(27, 27, 27), max_level=0, cfl=0.1,
                 gamma=1.4, picard_iters=0, precision="fp64", lo=(0.0, 0.0, 0.0),
                 hi=(1.0, 1.0, 1.0), device=None, predictor="picard", limiter=False,
                 limiter_delta0=1e-4, limiter_eps=1e-3, pipeline_chunks=0,
                 pipeline_ctas=0, eager_steps=False):
        import torch
        self.torch = torch
        self.device = torch.device("cuda" if device is None else device)
        cfg = A.ader_config()
        cfg.dim = dim
        cfg.order = order
        cfg.pde = A.ADER_EULER if pde == "euler" else A.ADER_ACOUSTICS
        cfg.nvar = dim + 2 if pde == "euler" else dim + 1
        cfg.gamma = gamma
        cfg.cfl = cfl
        for d in range(3):
            cfg.base[d] = base[d] if d < dim else 1
            cfg.lo[d] = lo[d] if d < dim else 0.0
            cfg.hi[d] = hi[d] if d < dim else 1.0
        cfg.max_level = max_level
        cfg.picard_iters = picard_iters
        cfg.prec = A.PRECISIONS[precision]
        cfg.predictor = A.ADER_PREDICTOR_CK if predictor == "ck" else A.ADER_PREDICTOR_PICARD
        cfg.limiter = 1 if limiter else 0
        cfg.limiter_delta0 = limiter_delta0
        cfg.limiter_eps = limiter_eps
        cfg.pipeline_chunks = pipeline_chunks
        cfg.pipeline_ctas = pipeline_ctas
        cfg.eager_steps = 1 if eager_steps else 0
        self.cfg = cfg
        self.dim, self.order, self.n, self.nvar = dim, order, order + 1, cfg.nvar
        with torch.cuda.device(self.device):
            self.ctx = A.ader_init(cfg)
            self.dt = torch.zeros(1, dtype=torch.float64, device=self.device)

    # ------------------------------------------------------------------ mesh
    @property
    def ncells(self):
        return A.ader_mesh_info(self.ctx)[0]

    def mesh_info(self):
        return A.ader_mesh_info(self.ctx)

    def cells(self):
        return A.ader_mesh_cells(self.ctx)

    def skeleton(self):
        return A.ader_mesh_skeleton(self.ctx)

    def nodes(self):
        return A.ader_nodes(self.ctx, self.n)

    def state_shape(self):
        return (self.ncells, self.nvar) + (self.n,) * self.dim

    def node_coords(self):
        """Physical node coordinates per direction, arrays (C, *nodes)."""
        cells = self.cells()
        xi = self.nodes()
        out = []
        C = len(cells)
        for d in range(self.dim):
            L = self.cfg.hi[d] - self.cfg.lo[d]
            h = L / (self.cfg.base[d] * 3.0 ** cells[:, 0])
            org = self.cfg.lo[d] + cells[:, 1 + d] * h
            shape = [1] * self.dim
            shape[self.dim - 1 - d] = self.n
            v = org.reshape((C,) + (1,) * self.dim) + h.reshape((C,) + (1,) * self.dim) * \
                xi.reshape(shape)
            out.append(np.broadcast_to(v, (C,) + (self.n,) * self.dim).copy())
        return out

    # ----------------------------------------------------------------- state
    def _stream(self, stream):
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def set_state(self, u, stream=None):
        torch = self.torch
        if isinstance(u, np.ndarray):
            u = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float64))
        assert tuple(u.shape) == self.state_shape(), (u.shape, self.state_shape())
        u = u.contiguous()
        A.ader_set_state(self.ctx, u.data_ptr(), u.is_cuda, self._stream(stream))
        if u.is_cuda:
            self.torch.cuda.current_stream(self.device).synchronize()

    def get_state(self, stream=None):
        out = self.torch.empty(self.state_shape(), dtype=self.torch.float64, device=self.device)
        A.ader_get_state(self.ctx, out.data_ptr(), True, self._stream(stream))
        return out

    def get_field(self, field, stream=None):
        C, m, n, d = self.ncells, self.nvar, self.n, self.dim
        if field in (A.ADER_FIELD_U, A.ADER_FIELD_USTAR):
            shape = self.state_shape()
        else:
            shape = (C, d, 2, m, n ** (d - 1))
        out = self.torch.empty(shape, dtype=self.torch.float64, device=self.device)
        A.ader_get_field(self.ctx, field, out.data_ptr(), True, self._stream(stream))
        return out

    # ------------------------------------------------------------------ step
    def set_dt(self, dt):
        self.dt.fill_(float(dt))

    def compute_dt(self, stream=None):
        A.ader_compute_dt(self.ctx, self.dt.data_ptr(), self._stream(stream))
        return self.dt

    def predict(self, which=A.ADER_ALL, stream=None):
        A.ader_predict(self.ctx, self.dt.data_ptr(), which, self._stream(stream))

    def riemann(self, which=A.ADER_ALL, stream=None):
        A.ader_riemann(self.ctx, which, self._stream(stream))

    def correct(self, dt_next=None, stream=None):
        out = self.dt if dt_next is None else dt_next
        A.ader_correct(self.ctx, self.dt.data_ptr(), out.data_ptr(), self._stream(stream))

    def step(self, nsteps=1, stream=None):
        A.ader_step(self.ctx, nsteps, self.dt.data_ptr(), self._stream(stream))

    def step_fixed_dt(self, nsteps=1, dt_next=None, stream=None):
        """nsteps steps with the prescribed dt in ``self.dt`` (the shifted
        task graph: corrector and next predictor as one pass per cell); the
        final state's CFL time step goes to ``dt_next`` (a device scalar)
        when given."""
        A.ader_step_fixed_dt(self.ctx, nsteps, self.dt.data_ptr(),
                             None if dt_next is None else dt_next.data_ptr(), self._stream(stream))

    def remesh(self, flags):
        A.ader_remesh(self.ctx, flags)

    def classify(self, flags=None):
        A.ader_classify(self.ctx, flags)

    def gradient_flags(self, var, refine_above, coarsen_below, deriv=1):
        """(eta, flags): eta = h |grad q| (deriv 1) or h^2 |Hessian q|_F
        (deriv 2) per cell, q = variable ``var``."""
        return A.ader_gradient_flags(self.ctx, var, refine_above, coarsen_below, deriv)

    def gradient_indicator(self, var, stream=None, deriv=1):
        """Device tensor eta[c] of gradient_flags, enqueued on ``stream``."""
        eta = self.torch.empty(self.ncells, dtype=self.torch.float64, device=self.device)
        A.ader_gradient_indicator(self.ctx, var, eta, self._stream(stream), deriv)
        return eta

    def sphere_flags(self, center, radius):
        return A.ader_sphere_flags(self.ctx, center, radius)

    def status(self):
        return A.ader_status_word(self.ctx)

    def launch_count(self):
        return A.ader_launch_count(self.ctx)

    # --------------------------------------------------------------- limiter
    def limiter_flags(self):
        """(flags per cell, number of limited cells) of the last corrector:
        bit 0 limited, bit 1 face flux replaced, bit 2 kept at a transition."""
        return A.ader_limiter_flags(self.ctx, self._stream(None))

    def limiter_refine_flags(self):
        """Remesh flags that refine around the last step's troubled cells."""
        return A.ader_limiter_refine_flags(self.ctx)

    def step_refining(self, max_rounds=2, stream=None):
        """One limited step; troubled cells at resolution transitions make the
        context refine around them and redo the step from u(T).  Returns the
        number of refinements."""
        return A.ader_step_refining(self.ctx, self.dt, max_rounds, self._stream(stream))

    def force_limit(self, mask):
        """Treat the cells in ``mask`` as troubled in the following steps
        (None clears)."""
        A.ader_limiter_force(self.ctx, mask)

    def close(self):
        if getattr(self, "ctx", None):
            A.ader_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
