"""Cell and face tasks of one ADER-DG step (oracle; test infrastructure).

Sec. 2.1-2.2 and Eq. (4) of the paper split one step into the space-time
predictor C_STP with its projections id|dc (onto the 2d faces) and id|T+dT,
the Riemann solves F_R over the faces, and the corrector C_Corr.  The paper
defers the formulas to the ADER-DG literature; this module writes them out for
a nodal Gauss-Legendre basis on cells of widths h_d, reference time
tau in [0, 1] with t = T + tau dt.

Array layout: a cell batch is ``u[c, var, *nodes]`` with the node axes ordered
(z, y, x) in 3D and (y, x) in 2D, so direction ``dr`` (0 = x) is array axis
``u.ndim - 1 - dr``.  A face array flattens the remaining node axes in C order
(lowest tangential direction fastest).  ``h`` has shape (C, d).

Readings where the paper is silent (each listed in the design notes):

* the predictor keeps the spatial flux divergence in strong (nodal
  derivative) form, because it "drops all jump terms" and ignores neighbours;
* the predictor runs a fixed number of Picard iterations (default N + 1);
* the face flux F-bar is the time average of the flux of the final iterate;
* Riemann solves act on time-averaged face data (Algorithm 1's caption allows
  collapsing the time integral into one spatial Riemann problem), with one
  Rusanov speed per face: the largest lambda_d over both sides' face nodes.
"""
import math

import numpy as np

from .basis import apply_axis, contract_axis


def node_axis(ndim_array, dr):
    return ndim_array - 1 - dr


def _bcast(v, ndim):
    """Reshape a per-cell vector (C,) to broadcast against an ndim array."""
    return np.reshape(v, (-1,) + (1,) * (ndim - 1))


def _flux_var_axis(pde, q, dr, var_axis):
    f = pde.flux(np.moveaxis(q, var_axis, 0), dr)
    return np.moveaxis(f, 0, var_axis)


def divergence(pde, q, h, D, var_axis):
    """sum_d h_d^-1 D^(d) f_d(q): strong-form nodal flux divergence."""
    dim = h.shape[1]
    out = np.zeros_like(q)
    for dr in range(dim):
        f = _flux_var_axis(pde, q, dr, var_axis)
        out += apply_axis(D, f, node_axis(q.ndim, dr)) / _bcast(h[:, dr], q.ndim)
    return out


def picard_predictor(u, h, dt, pde, B, iters):
    """Space-time predictor C_STP by Picard iteration (Sec. 2.1).

    For every spatial node i and time node k the predictor solves
        sum_l K1[k, l] q[l, i] = theta_k(0) u_i - dt w_k (sum_d h_d^-1 D^(d) f_d(q_k))_i
    starting from q^(0)[k] = u.  Each iteration evaluates the right-hand side at
    the current iterate and solves with K1 along time.  Returns q with shape
    (C, n_t, m, *nodes).
    """
    n = B.n
    q = np.repeat(u[:, np.newaxis], n, axis=1)
    theta0 = B.phi0.reshape((1, n) + (1,) * (u.ndim - 1))
    wt = B.w.reshape((1, n) + (1,) * (u.ndim - 1))
    for _ in range(iters):
        div = divergence(pde, q, h, B.D, var_axis=2)
        rhs = theta0 * u[:, np.newaxis] - dt * wt * div
        rhs_t = np.moveaxis(rhs, 1, 0)
        sol = np.linalg.solve(B.K1, rhs_t.reshape(n, -1)).reshape(rhs_t.shape)
        q = np.moveaxis(sol, 0, 1)
    return q


def ck_predictor(u, h, dt, pde, B):
    """Cauchy-Kowalevski predictor for a linear PDE (Sec. 2.4).

    Time derivatives by the PDE itself: d_t^0 u = u and
    d_t^{k+1} u = -sum_d h_d^-1 D^(d) f_d(d_t^k u) (f linear).  The space-time
    polynomial is the Taylor series q(tau) = sum_{k<=N} (tau dt)^k / k! d_t^k u,
    evaluated at the time nodes.  Returns q with shape (C, n_t, m, *nodes).
    """
    assert pde.linear
    derivs = [u]
    for _ in range(B.order):
        derivs.append(-divergence(pde, derivs[-1], h, B.D, var_axis=1))
    q = np.zeros((u.shape[0], B.n) + u.shape[1:])
    for k in range(B.n):
        tau = B.xi[k]
        for j, dj in enumerate(derivs):
            q[:, k] += (tau * dt) ** j / math.factorial(j) * dj
    return q


def time_average(q, pde, B):
    """Q-bar = sum_k w_k q_k and F-bar_d = sum_k w_k f_d(q_k) (id|T+dT side data)."""
    dim = q.ndim - 3
    qbar = contract_axis(B.w, q, 1)
    fbar = []
    for dr in range(dim):
        f = _flux_var_axis(pde, q, dr, var_axis=2)
        fbar.append(contract_axis(B.w, f, 1))
    return qbar, fbar


def volume_update(u, fbar, h, dt, B):
    """u* = u + dt sum_d h_d^-1 w_{i_d}^-1 sum_j w_j D[j, i_d] F-bar_d(.., j, ..).

    The volume part of the corrector: the weak form integrated by parts in
    space (Sec. 2.1 advantage (ii)), with the diagonal GL mass matrix.
    """
    V = (B.D.T * B.w[np.newaxis, :]) / B.w[:, np.newaxis]
    out = u.copy()
    for dr, f in enumerate(fbar):
        out += dt * apply_axis(V, f, node_axis(u.ndim, dr)) / _bcast(h[:, dr], u.ndim)
    return out


def face_values(x, dr, side, B):
    """Extrapolate a cell field x[c, var, *nodes] to its face (dr, side).

    side 0 is the face at xi_dr = 0, side 1 the face at xi_dr = 1.  Returns
    [c, var, n^(d-1)] (remaining node axes flattened in C order).
    """
    phi = B.phi0 if side == 0 else B.phi1
    y = contract_axis(phi, x, node_axis(x.ndim, dr))
    return y.reshape(y.shape[0], y.shape[1], -1)


def project_to_faces(qbar, fbar, B):
    """id|dc: face data Q-bar and the normal flux F-bar_d on all 2d faces.

    Returns Qf, Ff of shape (C, d, 2, m, n^(d-1)).
    """
    dim = len(fbar)
    C, m = qbar.shape[:2]
    nf = B.n ** (dim - 1)
    Qf = np.empty((C, dim, 2, m, nf))
    Ff = np.empty((C, dim, 2, m, nf))
    for dr in range(dim):
        for side in range(2):
            Qf[:, dr, side] = face_values(qbar, dr, side, B)
            Ff[:, dr, side] = face_values(fbar[dr], dr, side, B)
    return Qf, Ff


def rusanov(QL, FL, QR, FR, pde, dr):
    """Rusanov flux F* = (F_L + F_R)/2 - s (Q_R - Q_L)/2 on faces [f, var, node].

    s is one estimate of the largest eigenvalue per face (Sec. 2.4): the
    maximum of lambda_dr over the face nodes of both sides.
    """
    lamL = pde.max_speed(np.moveaxis(QL, 1, 0), dr)
    lamR = pde.max_speed(np.moveaxis(QR, 1, 0), dr)
    s = np.maximum(lamL.max(axis=-1), lamR.max(axis=-1))
    return 0.5 * (FL + FR) - 0.5 * s[:, np.newaxis, np.newaxis] * (QR - QL)


def face_lifting(ustar, Fs, h, dt, B):
    """Corrector face part: u = u* + dt sum_d h_d^-1 w_{i_d}^-1
    [-phi_{i_d}(1) F*_{d,+} + phi_{i_d}(0) F*_{d,-}] (Fs: (C, d, 2, m, nf))."""
    dim = Fs.shape[1]
    n = B.n
    out = ustar.copy()
    C, m = ustar.shape[:2]
    for dr in range(dim):
        ax = node_axis(ustar.ndim, dr)
        shape_vec = [1] * ustar.ndim
        shape_vec[ax] = n
        for side, sign, phi in ((0, 1.0, B.phi0), (1, -1.0, B.phi1)):
            face = Fs[:, dr, side].reshape((C, m) + (n,) * (dim - 1))
            face = np.expand_dims(face, ax)
            lift = (sign * phi / B.w).reshape(shape_vec)
            out += dt * face * lift / _bcast(h[:, dr], ustar.ndim)
    return out


def cfl_rate(u, h, pde):
    """max over cells and nodes of sum_d lambda_d(u) / h_d."""
    dim = h.shape[1]
    q = np.moveaxis(u, 1, 0)
    rate = np.zeros(u.shape[:1] + u.shape[2:])
    for dr in range(dim):
        rate = rate + pde.max_speed(q, dr) / _bcast(h[:, dr], rate.ndim)
    return rate.max()


def cfl_dt(u, h, pde, order, cfl=None):
    """Global time step dt = C / max_c max_nodes sum_d lambda_d / h_d (global
    time stepping, Sec. 2.1).  By default C = 0.9 nu_N with nu_N the
    one-dimensional linear stability limit of this scheme (``stability``)."""
    if cfl is None:
        from .stability import cfl_number
        cfl = cfl_number(order)
    return cfl / cfl_rate(u, h, pde)


def prolong_face(x, s, B, dim):
    """Interpolate face data x[..., var, nf] of a coarse face onto its child
    sub-face s = (s_t for each tangential direction, lowest first)."""
    n = B.n
    lead = x.shape[:-1]
    y = x.reshape(lead + (n,) * (dim - 1))
    for t, st in enumerate(s):
        y = apply_axis(B.P[st], y, y.ndim - 1 - t)
    return y.reshape(lead + (-1,))


def restrict_face(x, s, B, dim):
    """Mass-weighted transpose of ``prolong_face``: child sub-face s -> parent."""
    n = B.n
    lead = x.shape[:-1]
    y = x.reshape(lead + (n,) * (dim - 1))
    for t, st in enumerate(s):
        y = apply_axis(B.R[st], y, y.ndim - 1 - t)
    return y.reshape(lead + (-1,))


def prolong_volume(x, s, B):
    """Interpolate a cell field x[c, var, *nodes] into child s = (s_x, s_y[, s_z])."""
    y = x
    for dr, sd in enumerate(s):
        y = apply_axis(B.P[sd], y, node_axis(y.ndim, dr))
    return y


def restrict_volume(x, s, B):
    """Mass-weighted transpose of ``prolong_volume`` for child s."""
    y = x
    for dr, sd in enumerate(s):
        y = apply_axis(B.R[sd], y, node_axis(y.ndim, dr))
    return y


def cell_integral(u, h, B):
    """sum_c prod_d h_{c,d} sum_i W_i u_i per variable (GL quadrature)."""
    dim = h.shape[1]
    y = u
    for _ in range(dim):
        y = contract_axis(B.w, y, y.ndim - 1)
    vol = np.prod(h, axis=1)
    return (y * vol[:, np.newaxis]).sum(axis=0)
