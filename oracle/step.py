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


def predict(u, h, dt, pde, B, iters, predictor="picard"):
    """C_STP followed by id|T+dT and id|dc, plus the corrector's volume term.
    ``predictor`` selects Picard iteration or, for a linear PDE, the
    Cauchy-Kowalevski Taylor expansion (Sec. 2.4)."""
    if predictor == "ck":
        q = ader.ck_predictor(u, h, dt, pde, B)
    else:
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


def step(mesh, u, dt, pde, B, iters=None, predictor="picard"):
    if iters is None:
        iters = B.order + 1
    h = mesh.cell_widths()
    ustar, Qf, Ff = predict(u, h, dt, pde, B, iters, predictor)
    Fs = riemann(mesh, Qf, Ff, pde, B)
    unew, dt_next = correct(ustar, Fs, h, dt, pde, B)
    return StepOutput(unew, ustar, Qf, Ff, Fs, dt_next)


def step_sample(mesh, u, dt, pde, B, targets, iters=None):
    """u(T + dt) of one full step for the cells ``targets`` only.

    The same tasks as ``step`` evaluated cell by cell: the predictor on the
    targets and on every cell that shares a face with them (conforming
    neighbours, finer cells across a parent face, the coarser cell across a
    child face), the Riemann solves on the targets' faces (prolongation to the
    virtual face, and restriction of all child faces of a target's parent
    face), and the corrector on the targets.  Returns (len(targets), m, *nodes).
    """
    if iters is None:
        iters = B.order + 1
    dim = mesh.dim
    need = set(int(t) for t in targets)
    plan = []          # per target: list of (dr, side, kind, data)
    for t in targets:
        key = mesh.cells[int(t)]
        faces = []
        for dr in range(dim):
            for side in range(2):
                nb = mesh.neighbor(key, dr, side)
                if nb in mesh.leaves:
                    j = mesh.index[nb]
                    need.add(j)
                    faces.append((dr, side, "conf", j))
                elif nb in mesh.refined:
                    kids = mesh.touching_children(nb, dr, 1 - side)
                    idx = [(mesh.index[ck], s) for ck, s in kids]
                    need.update(j for j, _ in idx)
                    faces.append((dr, side, "parent", idx))
                else:
                    coarse = nb
                    while coarse not in mesh.leaves:
                        coarse = (coarse[0] - 1, tuple(c // 3 for c in coarse[1]))
                    j = mesh.index[coarse]
                    need.add(j)
                    s = tuple(key[1][a] - 3 * coarse[1][a] for a in range(dim) if a != dr)
                    faces.append((dr, side, "child", (j, s)))
        plan.append(faces)
    sub = sorted(need)
    pos = {c: i for i, c in enumerate(sub)}
    h_all = mesh.cell_widths()
    ustar, Qf, Ff = predict(u[sub], h_all[sub], dt, pde, B, iters)

    def rus(dr, L, R):
        (QL, FL), (QR, FR) = L, R
        return ader.rusanov(QL[None], FL[None], QR[None], FR[None], pde, dr)[0]

    out = []
    for t, faces in zip(targets, plan):
        i = pos[int(t)]
        Fs = np.zeros((1,) + Qf.shape[1:])
        for dr, side, kind, data in faces:
            mine = (Qf[i, dr, side], Ff[i, dr, side])
            if kind == "conf":
                j = pos[data]
                other = (Qf[j, dr, 1 - side], Ff[j, dr, 1 - side])
                Fs[0, dr, side] = rus(dr, mine, other) if side == 1 else rus(dr, other, mine)
            elif kind == "parent":
                acc = np.zeros(Qf.shape[3:])
                for j, s in data:
                    fine = (Qf[pos[j], dr, 1 - side], Ff[pos[j], dr, 1 - side])
                    virt = (ader.prolong_face(mine[0], s, B, dim), ader.prolong_face(mine[1], s, B, dim))
                    F = rus(dr, virt, fine) if side == 1 else rus(dr, fine, virt)
                    acc += ader.restrict_face(F[None], s, B, dim)[0]
                Fs[0, dr, side] = acc
            else:
                j, s = data
                jj = pos[j]
                cq, cf = Qf[jj, dr, 1 - side], Ff[jj, dr, 1 - side]
                virt = (ader.prolong_face(cq, s, B, dim), ader.prolong_face(cf, s, B, dim))
                Fs[0, dr, side] = rus(dr, mine, virt) if side == 1 else rus(dr, virt, mine)
        unew = ader.face_lifting(ustar[i:i + 1], Fs, h_all[[int(t)]], dt, B)
        out.append(unew[0])
    return np.stack(out)
