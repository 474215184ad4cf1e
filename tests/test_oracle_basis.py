"""Pins of the oracle's one-dimensional operators against closed forms."""
import math

import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_legendre_exactness(n):
    xi, w = basis.gauss_legendre01(n)
    for k in range(2 * n):
        assert abs(np.dot(w, xi ** k) - 1.0 / (k + 1)) < 1e-14
    # one degree beyond exactness the error is the closed-form GL remainder
    # (n!)^4 / ((2n+1) ((2n)!)^2) for x^(2n) on [0, 1]
    err = 1.0 / (2 * n + 1) - np.dot(w, xi ** (2 * n))
    exact = math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
    assert abs(err - exact) < 1e-14
    assert np.allclose(xi + xi[::-1], 1.0, atol=1e-15, rtol=0)
    assert np.all(np.diff(xi) > 0) and np.all(xi > 0) and np.all(xi < 1)


@pytest.mark.parametrize("N", range(1, 9))
def test_lagrange_and_derivative(N):
    xi, _ = basis.gauss_legendre01(N + 1)
    L = basis.lagrange(xi, xi)
    assert np.allclose(L, np.eye(N + 1), atol=1e-13, rtol=0)
    x = np.linspace(0.0, 1.0, 17)
    assert np.allclose(basis.lagrange(xi, x).sum(axis=1), 1.0, atol=1e-12, rtol=0)
    D = basis.derivative_matrix(xi)
    assert np.allclose(D @ np.ones(N + 1), 0.0, atol=1e-11, rtol=0)
    for k in range(1, N + 1):
        assert np.allclose(D @ xi ** k, k * xi ** (k - 1), atol=1e-10 * (N + 1) ** 2, rtol=0)
    phi0, phi1 = basis.extrapolation(xi)
    for k in range(N + 1):
        assert abs(phi0 @ xi ** k - (1.0 if k == 0 else 0.0)) < 1e-12
        assert abs(phi1 @ xi ** k - 1.0) < 1e-12


def pade_exp(N, z):
    """Closed-form (N, N+1) Pade approximant of exp(z)."""
    num = sum(math.factorial(2 * N + 1 - j) * math.factorial(N)
              / (math.factorial(2 * N + 1) * math.factorial(j) * math.factorial(N - j)) * z ** j
              for j in range(N + 1))
    den = sum(math.factorial(2 * N + 1 - j) * math.factorial(N + 1)
              / (math.factorial(2 * N + 1) * math.factorial(j) * math.factorial(N + 1 - j)) * (-z) ** j
              for j in range(N + 2))
    return num / den


@pytest.mark.parametrize("N", range(1, 9))
def test_time_matrix_is_dg_in_time(N):
    """K1 is DG in time with upwind inflow: for y' = z y its end value is the
    subdiagonal (N, N+1) Pade approximant of exp(z) (Radau IIA stability
    function), and K1 . 1 = theta(0)."""
    B = basis.Basis(N)
    assert np.allclose(B.K1 @ np.ones(B.n), B.phi0, atol=1e-12, rtol=0)
    for z in (-0.7, -0.1, 0.3, 1.1):
        q = np.linalg.solve(B.K1 - z * np.diag(B.w), B.phi0)
        assert abs(B.phi1 @ q - pade_exp(N, z)) < 1e-12
        # and it is close to exp(z) with the superconvergent order 2N+1
        assert abs(B.phi1 @ q - math.exp(z)) < 10.0 * abs(z) ** (2 * N + 2) / math.factorial(2 * N + 1) + 1e-14


@pytest.mark.parametrize("N", range(1, 9))
def test_prolongation_restriction(N):
    B = basis.Basis(N)
    for s in range(3):
        for k in range(N + 1):
            assert np.allclose(B.P[s] @ B.xi ** k, ((s + B.xi) / 3.0) ** k, atol=1e-11, rtol=0)
    acc = sum(B.R[s] @ B.P[s] for s in range(3))
    assert np.allclose(acc, np.eye(B.n), atol=1e-12, rtol=0)
    x = np.random.default_rng(N).standard_normal(B.n)
    for s in range(3):
        # restriction keeps the integral: int_parent R_s x = (1/3) int_child x
        assert abs(B.w @ (B.R[s] @ x) - (B.w @ x) / 3.0) < 1e-13
    # restriction of a polynomial restricted from its three children is exact:
    # child data of p on the children, projected back, gives p
    p = B.xi ** N - 0.3 * B.xi
    kids = [B.P[s] @ p for s in range(3)]
    assert np.allclose(sum(B.R[s] @ kids[s] for s in range(3)), p, atol=1e-12, rtol=0)


@pytest.mark.parametrize("N", range(1, 9))
def test_derivative_matrix_two_formulas(N):
    """The barycentric D agrees with the product-rule derivative of phi_j."""
    xi, _ = basis.gauss_legendre01(N + 1)
    D = basis.derivative_matrix(xi)
    assert np.allclose(D, basis.lagrange_deriv(xi, xi), atol=1e-11 * (N + 1) ** 2, rtol=0)
    assert np.abs(D.sum(axis=1)).max() < 1e-12
