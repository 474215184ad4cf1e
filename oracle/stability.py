"""Linear stability limit of the ADER-DG step per order (oracle; test
infrastructure).

The paper uses global time stepping with an admissible step size but gives no
CFL rule.  The rule used here is dt = C / max_c max_nodes sum_d lambda_d / h_d
with C = 0.9 nu_N, where nu_N is the von Neumann limit of the scheme itself:
the largest Courant number nu = dt a / h for which the one-dimensional step
(linear advection u_t + a u_x = 0, a > 0, upwind flux = Rusanov, N + 1 Picard
iterations, which are exact for this problem) has an amplification matrix
G(nu, theta) with spectral radius <= 1 (to 1e-4) for all Fourier angles theta.

G is assembled from the same one-dimensional operators as the oracle's step:
time average of the predictor, weak volume term, and face lifting with the
left neighbour's face value carried by exp(-i theta).
"""
import functools

import numpy as np

from .basis import Basis


def amplification(N, nu, theta, iters=None):
    return _parts(N, nu, iters)(theta)


def _parts(N, nu, iters=None):
    B = Basis(N)
    n = B.n
    if iters is None:
        iters = N + 1

    def predictor(u):
        q = np.tile(u, (n, 1))                       # q[k, i]
        for _ in range(iters):
            rhs = np.outer(B.phi0, u) - nu * B.w[:, None] * (q @ B.D.T)
            q = np.linalg.solve(B.K1, rhs)
        return q

    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = B.w @ predictor(e)                 # u -> time-averaged Q-bar
    V = (B.D.T * B.w[None, :]) / B.w[:, None]
    right = B.phi1 @ A                               # Q-bar at the cell's right face
    local = np.eye(n) + nu * (V @ A - np.outer(B.phi1 / B.w, right))
    left = nu * np.outer(B.phi0 / B.w, right)
    return lambda theta: local + np.exp(-1j * theta) * left


def spectral_radius(N, nu, n_theta=361):
    G = _parts(N, nu)
    return max(np.abs(np.linalg.eigvals(G(th))).max()
               for th in np.linspace(0.0, 2.0 * np.pi, n_theta))


@functools.lru_cache(maxsize=None)
def stability_limit(N, tol=1e-4, steps=24):
    """Bisection for nu_N on [0, 0.5]."""
    lo, hi = 0.0, 0.5
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        if spectral_radius(N, mid) <= 1.0 + tol:
            lo = mid
        else:
            hi = mid
    return lo


def cfl_number(N):
    """C = 0.9 nu_N, nu_N truncated to three decimals."""
    return 0.9 * np.floor(stability_limit(N) * 1000.0) / 1000.0
