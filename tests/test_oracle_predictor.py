"""Pins of the oracle's space-time predictor (Picard and Cauchy-Kowalevski)."""
import numpy as np
import pytest

from oracle import ader, basis, pde as pdes


def cell_coords(B, dim, h, origin):
    n = B.n
    out = []
    for dr in range(dim):
        shape = [1] * dim
        shape[dim - 1 - dr] = n
        out.append(np.broadcast_to(origin[dr] + h[dr] * B.xi.reshape(shape), (n,) * dim))
    return out


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 2), (3, 5)])
def test_free_stream_predictor(dim, N):
    """A constant state is the predictor's fixed point: q_k = u for all k."""
    B = basis.Basis(N)
    pde = pdes.Euler(dim)
    q0 = pde.primitive_to_conserved(1.2, [0.4, -0.3, 0.2][:dim], 0.8)
    u = np.broadcast_to(q0.reshape((1, -1) + (1,) * dim), (2, dim + 2) + (B.n,) * dim).copy()
    h = np.full((2, dim), 0.1)
    q = ader.picard_predictor(u, h, 0.9 / (2 * N + 1) * 0.1 / 5.0, pde, B, N + 1)
    assert np.allclose(q, u[:, None], atol=1e-14, rtol=0)


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_picard_entropy_wave_is_exact(N):
    """Euler data with uniform v and p and a density f(x) + g(y) with f, g
    polynomials of degree N, on a cell with h_x != h_y: the exact flow
    translates rho with v, a degree-N polynomial in time at every node, so the
    DG-in-time fixed point is exact and Picard reaches it in N + 1 iterations
    (a derivative scaled by the wrong cell width fails)."""
    B = basis.Basis(N)
    dim = 2
    pde = pdes.Euler(dim)
    h = np.array([[0.2, 0.3]])
    vx, vy, p = 0.7, -0.4, 1.3
    dt = 0.9 / (2 * N + 1) * 0.2 / 2.5      # the CFL step of the scheme
    cx, cy = np.random.default_rng(N).uniform(-0.1, 0.1, size=(2, N + 1))

    def rho_of(x, y):
        return 1.0 + sum(c * x ** k for k, c in enumerate(cx)) + sum(c * y ** k for k, c in enumerate(cy))

    X = cell_coords(B, dim, h[0], np.array([0.1, 0.0]))
    u = pde.primitive_to_conserved(rho_of(X[0], X[1]), [vx, vy], p)[np.newaxis]
    q = ader.picard_predictor(u, h, dt, pde, B, N + 1)
    for k in range(B.n):
        t = B.xi[k] * dt
        exact = pde.primitive_to_conserved(rho_of(X[0] - vx * t, X[1] - vy * t), [vx, vy], p)
        assert np.allclose(q[0, k], exact, atol=1e-13, rtol=0)


def dalembert_1d(p0, v0, x, t):
    """Exact 1D acoustics (c = 1) for initial functions p0, v0."""
    a = p0(x - t) + v0(x - t)
    b = p0(x + t) - v0(x + t)
    return 0.5 * (a + b), 0.5 * (a - b)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_picard_and_ck_match_dalembert(N):
    """Acoustics with data varying along x only and polynomial of degree N:
    the exact solution is d'Alembert's, a degree-N polynomial in t.  Both the
    CK Taylor predictor and Picard (N + 1 iterations) reproduce it."""
    B = basis.Basis(N)
    dim = 3
    pde = pdes.Acoustics(dim)
    rng = np.random.default_rng(100 + N)
    cp = rng.standard_normal(N + 1)
    cv = rng.standard_normal(N + 1)
    p0 = lambda x: sum(c * x ** k for k, c in enumerate(cp))
    v0 = lambda x: sum(c * x ** k for k, c in enumerate(cv))
    h = np.array([[0.5, 0.25, 0.125]])
    dt = 0.9 / (2 * N + 1) * 0.125 / 3.0
    X = cell_coords(B, dim, h[0], np.zeros(3))
    zero = np.zeros_like(X[0])
    u = np.stack([p0(X[0]), v0(X[0]), zero, zero])[np.newaxis]
    q_ck = ader.ck_predictor(u, h, dt, pde, B)
    q_pi = ader.picard_predictor(u, h, dt, pde, B, N + 1)
    for k in range(B.n):
        pe, ve = dalembert_1d(p0, v0, X[0], B.xi[k] * dt)
        for q in (q_ck, q_pi):
            assert np.allclose(q[0, k, 0], pe, atol=1e-12, rtol=0)
            assert np.allclose(q[0, k, 1], ve, atol=1e-12, rtol=0)
            assert np.allclose(q[0, k, 2:], 0.0, atol=1e-13, rtol=0)


def test_picard_vs_ck_general_data_rate():
    """General 3D acoustics data: Picard with dN + 1 iterations is the exact
    DG-in-time fixed point (one more iteration changes nothing), and it
    differs from the CK Taylor polynomial by O(dt^(N+2)) per unit time step."""
    N = 2
    B = basis.Basis(N)
    pde = pdes.Acoustics(3)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((2, 4) + (B.n,) * 3)
    h = np.full((2, 3), 0.5)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        q_pi = ader.picard_predictor(u, h, dt, pde, B, 3 * N + 1)
        q_more = ader.picard_predictor(u, h, dt, pde, B, 3 * N + 2)
        assert np.allclose(q_pi, q_more, atol=1e-14, rtol=0)
        q_ck = ader.ck_predictor(u, h, dt, pde, B)
        errs.append(np.abs(q_pi - q_ck).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > N + 0.7), rates


def test_time_average_and_faces_of_polynomial():
    """Time averages and face extrapolation of a space-time polynomial are
    exact integrals and end values."""
    N = 3
    B = basis.Basis(N)
    dim = 2
    pde = pdes.Acoustics(dim)
    X = cell_coords(B, dim, np.array([1.0, 1.0]), np.zeros(2))
    q = np.zeros((1, B.n, 3) + (B.n,) * dim)
    for k in range(B.n):
        t = B.xi[k]
        q[0, k, 0] = X[0] ** 2 * t ** 3 + X[1] * t
    qbar, fbar = ader.time_average(q, pde, B)
    assert np.allclose(qbar[0, 0], X[0] ** 2 / 4 + X[1] / 2, atol=1e-14)
    Qf, Ff = ader.project_to_faces(qbar, fbar, B)
    # x = 1 face (dr = 0, side 1): values at y nodes: 1/4 + y/2
    assert np.allclose(Qf[0, 0, 1, 0], 0.25 + B.xi / 2, atol=1e-14)
    # y = 0 face (dr = 1, side 0): x^2 / 4
    assert np.allclose(Qf[0, 1, 0, 0], B.xi ** 2 / 4, atol=1e-14)
    # F-bar_x of acoustics is (v_x, p, 0): the p part lands in variable 1
    assert np.allclose(Ff[0, 0, 1, 1], 0.25 + B.xi / 2, atol=1e-14)
