"""Solution-based refinement criterion (oracle; test infrastructure).

Sec. 2.4 describes the refinement criteria of the paper's code base as
studying first or second derivatives of the solution per cell.  Both forms,
on one variable q, with h_c = max_d h_d:

    first:   eta_c = max over the nodes of cell c of h_c |grad q|,
             |grad q|^2 = sum_d ((D^(d) q) / h_d)^2;
    second:  eta_c = max over the nodes of h_c^2 |H q|_F,
             |H q|_F^2 = sum_{a, b} ((D^(b) D^(a) q) / (h_a h_b))^2
             (the full Hessian, mixed entries included);

and the flag +1 (refine) if eta_c > refine_above and the cell is below the
finest level, -1 (coarsen) if eta_c < coarsen_below and above level 0,
0 otherwise.
"""
import numpy as np

from .basis import apply_axis


def _derivative(q, h, B, dr):
    """d/dx_dr of nodal data q[c, *nodes] (x fastest) on cells of widths h."""
    dim = h.shape[1]
    ax = q.ndim - 1 - dr
    return apply_axis(B.D, q, ax) / h[:, dr].reshape((-1,) + (1,) * dim)


def gradient_indicator(u, h, B, var, deriv=1):
    q = u[:, var]                                   # (C, *nodes)
    dim = h.shape[1]
    s2 = np.zeros_like(q)
    if deriv == 1:
        for dr in range(dim):
            dq = _derivative(q, h, B, dr)
            s2 = s2 + dq * dq
        weight = h.max(axis=1)
    elif deriv == 2:
        for a in range(dim):
            qa = _derivative(q, h, B, a)
            for b in range(dim):
                hab = _derivative(qa, h, B, b)
                s2 = s2 + hab * hab
        weight = h.max(axis=1) ** 2
    else:
        raise ValueError("deriv must be 1 or 2")
    eta = np.sqrt(s2).reshape(len(q), -1).max(axis=1)
    return eta * weight


def gradient_flags(mesh, u, B, var, refine_above, coarsen_below, deriv=1):
    eta = gradient_indicator(u, mesh.cell_widths(), B, var, deriv)
    flags = np.zeros(len(mesh.cells), dtype=np.int8)
    for i, k in enumerate(mesh.cells):
        if eta[i] > refine_above and k[0] < mesh.max_level:
            flags[i] = 1
        elif eta[i] < coarsen_below and k[0] > 0:
            flags[i] = -1
    return eta, flags
