"""Solution-based refinement criterion (oracle; test infrastructure).

Sec. 2.4 describes the refinement criteria of the paper's code base as
studying first or second derivatives of the solution per cell; here the
first-derivative form on one variable:

    eta_c = max over the nodes of cell c of h_c |grad q|,
    |grad q|^2 = sum_d ((D^(d) q) / h_d)^2,   h_c = max_d h_d,

and the flag +1 (refine) if eta_c > refine_above and the cell is below the
finest level, -1 (coarsen) if eta_c < coarsen_below and above level 0,
0 otherwise.
"""
import numpy as np

from .basis import apply_axis


def gradient_indicator(u, h, B, var):
    q = u[:, var]                                   # (C, *nodes)
    dim = h.shape[1]
    g2 = np.zeros_like(q)
    for dr in range(dim):
        ax = q.ndim - 1 - dr
        dq = apply_axis(B.D, q, ax) / h[:, dr].reshape((-1,) + (1,) * dim)
        g2 = g2 + dq * dq
    eta = np.sqrt(g2).reshape(len(q), -1).max(axis=1)
    return eta * h.max(axis=1)


def gradient_flags(mesh, u, B, var, refine_above, coarsen_below):
    eta = gradient_indicator(u, mesh.cell_widths(), B, var)
    flags = np.zeros(len(mesh.cells), dtype=np.int8)
    for i, k in enumerate(mesh.cells):
        if eta[i] > refine_above and k[0] < mesh.max_level:
            flags[i] = 1
        elif eta[i] < coarsen_below and k[0] > 0:
            flags[i] = -1
    return eta, flags
