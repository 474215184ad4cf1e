"""A posteriori subcell finite-volume limiter (oracle; test infrastructure).

Sec. 4 of the paper ("Finite Volumes") and its Euler experiments (Sec. 5-6):
ADER-DG computes a candidate solution; where the candidate is physically wrong
(a negative density, say) or oscillates, the cell's step is rolled back and
redone by a finite-volume scheme on a patch of (2N+1)^d subcells, a patch size
that keeps the FV time step of the same size as the DG one.  The paper reads
FV as ADER-DG with piecewise-constant shape functions and a degenerate
predictor whose update is the Riemann outcome alone, and takes the rest from
Dumbser, Zanotti, Loubere and Diot, J. Comput. Phys. 278 (2014).

Readings where the paper is silent:

* subcell data: the averages of the nodal polynomial over the S = 2N+1 equal
  subintervals of each direction (tensor product), v = A u with
  A[s, j] = mean of phi_j over [s/S, (s+1)/S];
* back to nodes: least squares, u = R v with R = (A^T A)^-1 A^T; it keeps the
  cell mean because constants lie in the nodal space;
* detection on the candidate u~ of the unlimited step: a non-finite value;
  for Euler, density or pressure <= 0 at a node or a subcell average; or the
  relaxed discrete maximum principle of Dumbser et al. on the subcell averages
  of every variable, min_V v^n - delta <= v~ <= max_V v^n + delta, where V is
  the cell and its conforming face neighbours and
  delta = max(1e-4, 1e-3 (max_V v^n - min_V v^n));
* FV step of a limited cell: one first-order Godunov-type update of size dt
  from u^n on the subcells, with the Rusanov flux and a local speed per
  subface, the halo being the adjacent subcell layer of each face neighbour at
  t^n (so a face between two limited cells gets the same flux from both);
* conservation at a face between a limited cell and an unlimited one: the
  unlimited cell's corrector lifts the L2 projection of the FV subface fluxes
  onto its face nodes, Pi[i, s] = A[s, i] / (S w_i), instead of its DG flux;
* one detection pass per step (an unlimited neighbour changed by that
  projection is not re-checked);
* no limiting across a resolution transition (the paper keeps adaptivity out
  of the FV regions): a troubled cell with a non-conforming face keeps its DG
  candidate and is reported as such;
* the next time step comes from the final state: the nodes of every cell and
  the subcell averages of the limited cells;
* refinement around the shocks (the paper refines the DG solution down to the
  FV level near shocks, so that no adaptivity cuts through an FV region):
  +1 for troubled cells and their face neighbours below the finest level, -1
  for every other cell above the base level.
"""
from dataclasses import dataclass

import numpy as np

from . import ader
from .basis import apply_axis, lagrange
from .step import step as dg_step

DELTA0 = 1e-4
EPS = 1e-3


class Subcells:
    """1D subcell operators for order N: A (S x n), R (n x S), Pi (n x S)."""

    def __init__(self, B):
        n, S = B.n, 2 * B.order + 1
        self.S = S
        A = np.zeros((S, n))
        for s in range(S):
            # GL quadrature with n points is exact for the degree-N basis
            A[s] = B.w @ lagrange(B.xi, (s + B.xi) / S)
        self.A = A
        self.R = np.linalg.solve(A.T @ A, A.T)
        self.Pi = A.T / (S * B.w[:, np.newaxis])


def averages(u, sc):
    """Subcell averages v[c, var, *subcells] of nodal data u[c, var, *nodes]."""
    v = u
    for ax in range(2, u.ndim):
        v = apply_axis(sc.A, v, ax)
    return v


def to_nodes(v, sc):
    """Least-squares nodal values from subcell averages."""
    u = v
    for ax in range(2, v.ndim):
        u = apply_axis(sc.R, u, ax)
    return u


def project_face(G, sc, dim):
    """Face fluxes G[var, S^(d-1)] on the subfaces -> face nodes [var, n^(d-1)]."""
    m = G.shape[0]
    y = G.reshape((m,) + (sc.S,) * (dim - 1))
    for ax in range(1, y.ndim):
        y = apply_axis(sc.Pi, y, ax)
    return y.reshape(m, -1)


def neighbors(mesh):
    """nb[c, dr, side]: the conforming face neighbour, or -1 across a
    resolution transition."""
    C = len(mesh.cells)
    nb = -np.ones((C, mesh.dim, 2), dtype=np.int64)
    for i, key in enumerate(mesh.cells):
        for dr in range(mesh.dim):
            for side in range(2):
                other = mesh.neighbor(key, dr, side)
                if other in mesh.leaves:
                    nb[i, dr, side] = mesh.index[other]
    return nb


def _admissible(pde, x):
    """Per cell: all values finite and, for Euler, rho > 0 and p > 0
    (x[c, var, *points])."""
    red = tuple(range(1, x.ndim))
    ok = np.isfinite(x).all(axis=red)
    if pde.name == "euler":
        q = np.moveaxis(x, 1, 0)
        with np.errstate(all="ignore"):
            p = pde.pressure(q)
        red_p = tuple(range(1, p.ndim))
        ok &= (q[0] > 0.0).all(axis=red_p) & (p > 0.0).all(axis=red_p)
    return ok


def detect(pde, u_old, u_cand, sc, nb, force=None):
    """Troubled cells of a candidate.  Returns (limited, kept): troubled cells
    that get the FV step, and troubled cells at a resolution transition that
    keep their DG candidate."""
    v_old = averages(u_old, sc)
    with np.errstate(all="ignore"):
        v_new = averages(u_cand, sc)
    red = tuple(range(2, v_old.ndim))
    mn, mx = v_old.min(axis=red), v_old.max(axis=red)          # (C, m)
    lo, hi = mn.copy(), mx.copy()
    for dr in range(nb.shape[1]):
        for side in range(2):
            j = nb[:, dr, side]
            has = j >= 0
            lo[has] = np.minimum(lo[has], mn[j[has]])
            hi[has] = np.maximum(hi[has], mx[j[has]])
    delta = np.maximum(DELTA0, EPS * (hi - lo))
    with np.errstate(invalid="ignore"):
        dmp = ((v_new.min(axis=red) < lo - delta) | (v_new.max(axis=red) > hi + delta)).any(axis=1)
    bad = dmp | ~_admissible(pde, u_cand) | ~_admissible(pde, v_new)
    if force is not None:
        bad |= np.asarray(force, dtype=bool)
    conforming = (nb >= 0).all(axis=(1, 2))
    return bad & conforming, bad & ~conforming


def rusanov_points(qL, qR, pde, dr):
    """Pointwise Rusanov flux between states q[var, ...] (local speed)."""
    s = np.maximum(pde.max_speed(qL, dr), pde.max_speed(qR, dr))
    return 0.5 * (pde.flux(qL, dr) + pde.flux(qR, dr)) - 0.5 * s * (qR - qL)


def fv_update(u_old, cells, nb, h, dt, pde, sc):
    """First-order FV step of size dt on the subcell patches of ``cells``.

    Returns (v_new, G): v_new[k] the new subcell averages of cells[k], and
    G[(c, dr, side)] the fluxes [var, S^(d-1)] through the subfaces of face
    (dr, side) of cell c (positive along +dr)."""
    S = sc.S
    v_old = averages(u_old, sc)
    v_new, G = [], {}
    for c in cells:
        v = v_old[c]                                   # (m, *S)
        dim = v.ndim - 1
        dv = np.zeros_like(v)
        for dr in range(dim):
            ax = v.ndim - 1 - dr
            left = np.take(v_old[nb[c, dr, 0]], [S - 1], axis=ax)
            right = np.take(v_old[nb[c, dr, 1]], [0], axis=ax)
            ext = np.concatenate([left, v, right], axis=ax)        # S + 2 layers
            qL = np.take(ext, np.arange(0, S + 1), axis=ax)
            qR = np.take(ext, np.arange(1, S + 2), axis=ax)
            F = rusanov_points(qL, qR, pde, dr)                    # S + 1 interfaces
            hs = h[c, dr] / S
            dv -= dt / hs * (np.take(F, np.arange(1, S + 1), axis=ax)
                             - np.take(F, np.arange(0, S), axis=ax))
            G[(int(c), dr, 0)] = np.take(F, 0, axis=ax).reshape(v.shape[0], -1)
            G[(int(c), dr, 1)] = np.take(F, S, axis=ax).reshape(v.shape[0], -1)
        v_new.append(v + dv)
    return np.stack(v_new) if v_new else np.zeros((0,) + v_old.shape[1:]), G


def _rate(x, h, pde):
    """max over points of sum_d lambda_d(x) / h_d, per cell (x[c, var, *points])."""
    q = np.moveaxis(x, 1, 0)
    r = np.zeros(x.shape[:1] + x.shape[2:])
    for dr in range(h.shape[1]):
        r = r + pde.max_speed(q, dr) / h[:, dr].reshape((-1,) + (1,) * (r.ndim - 1))
    return r.reshape(len(x), -1).max(axis=1)


@dataclass
class LimitedStep:
    u: np.ndarray          # final u(T + dt)
    candidate: object      # the unlimited step (StepOutput)
    limited: np.ndarray    # bool per cell: FV step taken
    kept: np.ndarray       # bool per cell: troubled at a transition, DG kept
    fixed: np.ndarray      # bool per cell: unlimited, face flux replaced by FV
    Fs: np.ndarray         # final face fluxes (C, d, 2, m, nf)
    dt_next: float


def step_limited(mesh, u, dt, pde, B, iters=None, force=None, predictor="picard", cfl=None):
    """One ADER-DG step followed by the a posteriori subcell FV limiter."""
    cand = dg_step(mesh, u, dt, pde, B, iters, predictor)
    sc = Subcells(B)
    nb = neighbors(mesh)
    h = mesh.cell_widths()
    limited, kept = detect(pde, u, cand.u, sc, nb, force)
    u_new = cand.u.copy()
    Fs = cand.Fs.copy()
    fixed = np.zeros(len(u), dtype=bool)
    T = np.flatnonzero(limited)
    v_lim, G = fv_update(u, T, nb, h, dt, pde, sc)
    if len(T):
        u_new[T] = to_nodes(v_lim, sc)
        for c in T:
            for dr in range(mesh.dim):
                for side in range(2):
                    D = nb[c, dr, side]
                    if not limited[D]:
                        Fs[D, dr, 1 - side] = project_face(G[(int(c), dr, side)], sc, mesh.dim)
                        fixed[D] = True
        Dl = np.flatnonzero(fixed)
        u_new[Dl] = ader.face_lifting(cand.ustar[Dl], Fs[Dl], h[Dl], dt, B)
    rate = _rate(u_new, h, pde).max()
    if len(T):
        rate = max(rate, _rate(v_lim, h[T], pde).max())
    if cfl is None:
        from .stability import cfl_number
        cfl = cfl_number(B.order)
    return LimitedStep(u_new, cand, limited, kept, fixed, Fs, cfl / rate)


def face_neighbours(mesh):
    """Face-neighbour leaves of every cell: the conforming neighbour, the finer
    cells across a parent face, the coarser cell across a child face."""
    conf, parents = mesh.faces()
    nb = [set() for _ in mesh.cells]
    for L, R, _ in conf:
        nb[L].add(R)
        nb[R].add(L)
    for coarse, _, _, kids in parents:
        for f, _ in kids:
            nb[coarse].add(f)
            nb[f].add(coarse)
    return nb


def refine_flags(mesh, troubled):
    """Remesh flags that bring troubled cells and their face neighbours to the
    finest level and coarsen everything else."""
    troubled = np.asarray(troubled, dtype=bool)
    mark = troubled.copy()
    nb = face_neighbours(mesh)
    for c in np.flatnonzero(troubled):
        for j in nb[c]:
            mark[j] = True
    flags = np.zeros(len(mesh.cells), dtype=np.int8)
    for i, (lvl, _) in enumerate(mesh.cells):
        if mark[i] and lvl < mesh.max_level:
            flags[i] = 1
        elif not mark[i] and lvl > 0:
            flags[i] = -1
    return flags
