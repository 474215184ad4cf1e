"""One ADER-DG time step on an adaptive mesh (oracle; test infrastructure).

Algorithm 1 of the paper (three task loops: predictor over all cells, Riemann
over all faces, corrector over all cells), extended by the two AMR tasks of
Sec. 2.3: interpolation of the coarse predictor into virtual cells ahead of
the Riemann solves on child faces, and restriction (accumulate-Riemann) of
the child results into the parent face ahead of the coarse corrector.
"""
from dataclasses import dataclass

import numpy as np

from . import ader
from .mesh import subface_indices


@dataclass
class StepOutput:
    u: np.ndarray        # u(T + dt)            (C, m, *nodes)
    ustar: np.ndarray    # u + volume term      (C, m, *nodes)
    Qf: np.ndarray       # face Q-bar           (C, d, 2, m, nf)
    Ff: np.ndarray       # face F-bar_d         (C, d, 2, m, nf)
    Fs: np.ndarray       # face F*              (C, d, 2, m, nf)
    dt_next: float


def predict(u, h, dt, pde, B, iters):
    """C_STP followed by id|T+dT and id|dc, plus the corrector's volume term."""
    q = ader.picard_predictor(u, h, dt, pde, B, iters)
    qbar, fbar = ader.time_average(q, pde, B)
    ustar = ader.volume_update(u, fbar, h, dt, B)
    Qf, Ff = ader.project_to_faces(qbar, fbar, B)
    return ustar, Qf, Ff


def riemann(mesh, Qf, Ff, pde, B):
    """F_R over all faces: conforming faces directly; parent faces by
    prolongation to the child faces, Rusanov there, and restriction."""
    dim = mesh.dim
    Fs = np.full_like(Qf, np.nan)
    conf, parents = mesh.faces()
    if conf:
        conf = np.asarray(conf, dtype=np.int64)
        for dr in range(dim):
            sel = conf[conf[:, 2] == dr]
            if len(sel) == 0:
                continue
            cL, cR = sel[:, 0], sel[:, 1]
            Fstar = ader.rusanov(Qf[cL, dr, 1], Ff[cL, dr, 1], Qf[cR, dr, 0], Ff[cR, dr, 0], pde, dr)
            Fs[cL, dr, 1] = Fstar
            Fs[cR, dr, 0] = Fstar
    for dr in range(dim):
        for cside in range(2):
            group = [p for p in parents if p[1] == dr and p[2] == cside]
            if not group:
                continue
            coarse = np.asarray([p[0] for p in group], dtype=np.int64)
            acc = np.zeros((len(group),) + Qf.shape[3:])
            for j, s in enumerate(subface_indices(dim, dr)):
                fine = np.asarray([p[3][j][0] for p in group], dtype=np.int64)
                assert all(p[3][j][1] == s for p in group)
                Qv = ader.prolong_face(Qf[coarse, dr, cside], s, B, dim)
                Fv = ader.prolong_face(Ff[coarse, dr, cside], s, B, dim)
                if cside == 1:   # coarse cell on the left of the face
                    Fstar = ader.rusanov(Qv, Fv, Qf[fine, dr, 0], Ff[fine, dr, 0], pde, dr)
                    Fs[fine, dr, 0] = Fstar
                else:            # coarse cell on the right
                    Fstar = ader.rusanov(Qf[fine, dr, 1], Ff[fine, dr, 1], Qv, Fv, pde, dr)
                    Fs[fine, dr, 1] = Fstar
                acc += ader.restrict_face(Fstar, s, B, dim)
            Fs[coarse, dr, cside] = acc
    return Fs


def correct(ustar, Fs, h, dt, pde, B):
    """C_Corr: face lifting onto u*, then the next global time step."""
    u = ader.face_lifting(ustar, Fs, h, dt, B)
    return u, ader.cfl_dt(u, h, pde, B.order)


def step(mesh, u, dt, pde, B, iters=None):
    if iters is None:
        iters = B.order + 1
    h = mesh.cell_widths()
    ustar, Qf, Ff = predict(u, h, dt, pde, B, iters)
    Fs = riemann(mesh, Qf, Ff, pde, B)
    unew, dt_next = correct(ustar, Fs, h, dt, pde, B)
    return StepOutput(unew, ustar, Qf, Ff, Fs, dt_next)
