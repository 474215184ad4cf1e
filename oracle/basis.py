"""Nodal basis on the reference interval [0, 1] (oracle; test infrastructure).

Sec. 2.1 of the paper represents Q_h in every cell as a linear combination of
Lagrange polynomials over Gauss-Legendre points, and develops it in time with
the same ansatz (tensor-product space-time polynomials).  This module builds the
one-dimensional ingredients of that ansatz from their definitions:

* ``gauss_legendre01``  - nodes xi_i and weights w_i on [0, 1] (sum w_i = 1);
* ``lagrange``          - phi_j(x) by the product formula;
* ``lagrange_deriv``    - phi_j'(x) by the product rule;
* ``derivative_matrix`` - D_ij = phi_j'(xi_i);
* ``time_matrix``       - K1_kl = theta_k(1) theta_l(1) - w_l D_lk, the matrix of
                          the time-weak predictor equation after integration by
                          parts in time with the upwind value q(0) = u;
* ``prolongation``      - P_s with (P_s)_ij = phi_j((s + xi_i) / 3), s = 0, 1, 2:
                          interpolation into the three children of 3-partitioning;
* ``restriction``       - R_s = (1/3) W^-1 P_s^T W, the mass-weighted transpose of
                          P_s (the "transpose of the interpolation" of Sec. 2.3,
                          read as the L2 projection so that it conserves).

All arithmetic is float64.
"""
import numpy as np


def gauss_legendre01(n):
    """n Gauss-Legendre nodes and weights mapped from [-1, 1] to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange(nodes, x):
    """L[p, j] = phi_j(x_p) for the Lagrange basis on ``nodes``."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                L[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return L


def lagrange_deriv(nodes, x):
    """L'[p, j] = phi_j'(x_p): product rule over the factors of phi_j."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    dL = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[m]))
            for k in range(n):
                if k != j and k != m:
                    term *= (x - nodes[k]) / (nodes[j] - nodes[k])
            dL[:, j] += term
    return dL


def derivative_matrix(nodes):
    """D[i, j] = phi_j'(xi_i): nodal values -> nodal values of the derivative.

    Barycentric form (Berrut and Trefethen, SIAM Review 2004, Sec. 9.3):
    D[i, j] = (lambda_j / lambda_i) / (xi_i - xi_j) for i != j with
    lambda_j = 1 / prod_{k != j} (xi_j - xi_k), and the diagonal chosen so that
    every row sums to zero (the derivative of a constant vanishes).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    lam = np.ones(n)
    for j in range(n):
        for k in range(n):
            if k != j:
                lam[j] /= nodes[j] - nodes[k]
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (lam[j] / lam[i]) / (nodes[i] - nodes[j])
        D[i, i] = -sum(D[i, j] for j in range(n) if j != i)
    return D


def time_matrix(nodes, weights):
    """K1[k, l] = theta_k(1) theta_l(1) - w_l D[l, k].

    Space-time predictor, time direction: test the time derivative with theta_k,
    integrate by parts over tau in [0, 1] and inject the known solution at
    tau = 0 (the upwind value, Sec. 2.1 advantage (i)).  The boundary term at
    tau = 1 gives theta_k(1) q(1); the volume term gives -int theta_k' q dtau,
    and with GL quadrature (exact here) int theta_k' theta_l = w_l theta_k'(xi_l).
    """
    phi1 = lagrange(nodes, 1.0)[0]
    D = derivative_matrix(nodes)
    return np.outer(phi1, phi1) - D.T * weights[np.newaxis, :]


def extrapolation(nodes):
    """(phi_j(0), phi_j(1)): values of the basis at the two ends of [0, 1]."""
    return lagrange(nodes, 0.0)[0], lagrange(nodes, 1.0)[0]


def prolongation(nodes):
    """P[s] with P[s][i, j] = phi_j((s + xi_i) / 3) for child s in {0, 1, 2}."""
    return np.stack([lagrange(nodes, (s + np.asarray(nodes)) / 3.0) for s in range(3)])


def restriction(nodes, weights):
    """R[s] = (1/3) W^-1 P[s]^T W, W = diag(w): L2 projection child -> parent."""
    P = prolongation(nodes)
    w = np.asarray(weights)
    return np.stack([(P[s].T * w[np.newaxis, :]) / (3.0 * w[:, np.newaxis]) for s in range(3)])


class Basis:
    """All one-dimensional matrices for polynomial order N (n = N + 1 nodes)."""

    def __init__(self, order):
        self.order = order
        self.n = order + 1
        self.xi, self.w = gauss_legendre01(self.n)
        self.D = derivative_matrix(self.xi)
        self.K1 = time_matrix(self.xi, self.w)
        self.phi0, self.phi1 = extrapolation(self.xi)
        self.P = prolongation(self.xi)
        self.R = restriction(self.xi, self.w)


def apply_axis(A, x, axis):
    """y[..., i, ...] = sum_j A[i, j] x[..., j, ...] along ``axis`` of x."""
    y = np.tensordot(A, x, axes=([1], [axis]))
    return np.moveaxis(y, 0, axis)


def contract_axis(v, x, axis):
    """y[...] = sum_j v[j] x[..., j, ...]: removes ``axis`` of x."""
    return np.tensordot(x, v, axes=([axis], [0]))
