"""Helpers for GPU parity tests: build the same adaptive mesh in the library
and in the oracle (same flag sequence, flags from the oracle), and map cells
between the two numberings by their (level, coordinates) keys."""
import numpy as np

from oracle import basis as obasis, mesh as omesh
import workloads


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0)


def rel_max(a, b):
    """Per-element bound: max |a - b| / max |b| (one wrong value among many
    cannot hide in the L2 norm of the whole field)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max() if b.size else 0.0
    return np.abs(a - b).max() / (den if den > 0 else 1.0) if b.size else 0.0


def close_fields(a, b, tol):
    """Relative L2 <= tol and the per-element bound <= 10 tol."""
    return rel_l2(a, b) < tol and rel_max(a, b) <= 10.0 * tol


def lib_keys(solver):
    cells = solver.cells()
    d = solver.dim
    return [(int(c[0]), tuple(int(x) for x in c[1:1 + d])) for c in cells]


def build_pair(dim, order, pde="euler", base=9, max_level=0, centers=(), radius=0.15,
               precision="fp64", picard_iters=0, cfl=None, predictor="picard", **solver_kw):
    from paper_1806_07984_gb300 import Solver
    solver = Solver(dim, order, pde, base=(base,) * 3, max_level=max_level,
                    cfl=workloads.ADER_CFL[order] if cfl is None else cfl,
                    precision=precision, picard_iters=picard_iters, predictor=predictor,
                    **solver_kw)
    om = omesh.Mesh(dim, (base,) * dim, max_level)
    B1 = obasis.Basis(1)
    for c in centers:
        fl = omesh.sphere_flags(om, c, radius)
        perm = [om.index[k] for k in lib_keys(solver)]
        solver.remesh(fl[perm])
        om.remesh(np.zeros((len(om.cells), 1) + (2,) * dim), fl, B1)
    keys = lib_keys(solver)
    assert sorted(keys) == om.cells
    perm = np.array([om.index[k] for k in keys])
    return solver, om, perm
