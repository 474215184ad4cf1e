"""Pins of the oracle's fluxes and of the Rusanov solver."""
import numpy as np
import pytest

from oracle import ader, pde as pdes
import workloads


def jacobian(pde, q, d):
    """Complex-step Jacobian of f_d at a single state q[var]."""
    m = len(q)
    J = np.zeros((m, m))
    eps = 1e-30
    for j in range(m):
        qc = q.astype(np.complex128)
        qc[j] += 1j * eps
        J[:, j] = pde.flux(qc, d).imag / eps
    return J


@pytest.mark.parametrize("dim", [2, 3])
def test_euler_eigenstructure(dim):
    """The Euler flux Jacobian has eigenvalues v_d - c, v_d (d-fold), v_d + c;
    the wave-speed estimate is the largest modulus."""
    pde = pdes.Euler(dim)
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = rng.uniform(0.5, 2.0)
        vel = rng.uniform(-1.0, 1.0, size=dim)
        p = rng.uniform(0.5, 2.0)
        q = pde.primitive_to_conserved(rho, vel, p)
        c = np.sqrt(1.4 * p / rho)
        for d in range(dim):
            ev = np.sort(np.linalg.eigvals(jacobian(pde, q, d)).real)
            expect = np.sort([vel[d] - c] + [vel[d]] * dim + [vel[d] + c])
            assert np.allclose(ev, expect, atol=1e-10)
            assert abs(pde.max_speed(q, d) - np.max(np.abs(expect))) < 1e-14


def test_euler_rest_state_and_rotation():
    pde = pdes.Euler(3)
    q = pde.primitive_to_conserved(1.3, [0.0, 0.0, 0.0], 2.0)
    for d in range(3):
        f = pde.flux(q, d)
        e = np.zeros(5)
        e[1 + d] = 2.0          # only the pressure acts at rest
        assert np.array_equal(f, e)
    # rotational invariance: swapping x and y velocity swaps the fluxes
    q = pde.primitive_to_conserved(0.9, [0.3, -0.7, 0.2], 1.1)
    perm = [0, 2, 1, 3, 4]
    fx = pde.flux(q, 0)
    fy_swapped = pde.flux(q[perm], 1)[perm]
    assert np.allclose(fx, fy_swapped, atol=1e-15)


def test_acoustics_eigenstructure():
    pde = pdes.Acoustics(3)
    for d in range(3):
        ev = np.sort(np.linalg.eigvals(pde.jacobian(d)).real)
        assert np.allclose(ev, [-1, 0, 0, 1])
        q = np.arange(4.0)
        assert np.array_equal(pde.flux(q, d), pde.jacobian(d) @ q)


@pytest.mark.parametrize("dim", [2, 3])
def test_rusanov_consistency(dim):
    """F*(q, q) = f(q) bit for bit, for Euler and acoustics."""
    rng = np.random.default_rng(5)
    nf = 9
    for pde, q in ((pdes.Euler(dim), workloads.random_euler(rng, dim, (7, nf))),
                   (pdes.Acoustics(dim), workloads.random_acoustics(rng, dim, (7, nf)))):
        q = np.moveaxis(q, 0, 1)            # (faces, var, nodes)
        for d in range(dim):
            f = np.moveaxis(pde.flux(np.moveaxis(q, 1, 0), d), 0, 1)
            assert np.array_equal(ader.rusanov(q, f, q, f, pde, d), f)


def test_rusanov_acoustics_is_godunov_on_normal_waves():
    """For acoustics with c = 1 the Rusanov speed is exact and the flux of
    (p, v_n) equals the Godunov flux from the characteristic (d'Alembert)
    states p* = (pL + pR)/2 - (vR - vL)/2, v* = (vL + vR)/2 - (pR - pL)/2."""
    pde = pdes.Acoustics(2)
    rng = np.random.default_rng(9)
    QL = rng.standard_normal((4, 3, 5))
    QR = rng.standard_normal((4, 3, 5))
    for d in range(2):
        FL = np.moveaxis(pde.flux(np.moveaxis(QL, 1, 0), d), 0, 1)
        FR = np.moveaxis(pde.flux(np.moveaxis(QR, 1, 0), d), 0, 1)
        F = ader.rusanov(QL, FL, QR, FR, pde, d)
        pL, pR = QL[:, 0], QR[:, 0]
        vL, vR = QL[:, 1 + d], QR[:, 1 + d]
        pstar = 0.5 * (pL + pR) - 0.5 * (vR - vL)
        vstar = 0.5 * (vL + vR) - 0.5 * (pR - pL)
        assert np.allclose(F[:, 0], vstar, atol=1e-14)
        assert np.allclose(F[:, 1 + d], pstar, atol=1e-14)


def test_rusanov_mirror_symmetry():
    """Reflecting x -> -x swaps the sides and flips the sign of the normal
    momentum and of the flux of every other variable."""
    pde = pdes.Euler(2)
    rng = np.random.default_rng(11)
    QL = np.moveaxis(workloads.random_euler(rng, 2, (6, 4)), 0, 1)
    QR = np.moveaxis(workloads.random_euler(rng, 2, (6, 4)), 0, 1)
    flip = np.array([1.0, -1.0, 1.0, 1.0])[None, :, None]

    def fl(q):
        return np.moveaxis(pde.flux(np.moveaxis(q, 1, 0), 0), 0, 1)

    F = ader.rusanov(QL, fl(QL), QR, fl(QR), pde, 0)
    Fm = ader.rusanov(QR * flip, fl(QR * flip), QL * flip, fl(QL * flip), pde, 0)
    assert np.allclose(F, -flip * Fm, atol=1e-14)


def test_rusanov_speed_bounds_every_wave_on_the_face():
    """Sec. 2.4: one estimate of the largest eigenvalue per face.  On Euler
    faces whose nodes carry different states, the dissipation coefficient
    implied by F* (from F* - (F_L + F_R)/2 = -s (Q_R - Q_L)/2) is one number per
    face, no smaller than any local wave speed |v_d| + c on either side (the
    bound a monotone local Lax-Friedrichs flux needs) and no larger than the
    largest of them."""
    dim, d = 3, 1
    pde = pdes.Euler(dim)
    rng = np.random.default_rng(13)
    QL = np.moveaxis(workloads.random_euler(rng, dim, (5, 9), amp=0.3), 0, 1)
    QR = np.moveaxis(workloads.random_euler(rng, dim, (5, 9), amp=0.3), 0, 1)
    QR[2, :, 4] = pde.primitive_to_conserved(1.0, [0.5, 3.0, 0.2], 1.0)   # one fast node, v_y = 3

    def fl(q):
        return np.moveaxis(pde.flux(np.moveaxis(q, 1, 0), d), 0, 1)

    F = ader.rusanov(QL, fl(QL), QR, fl(QR), pde, d)
    jump = QR - QL
    ok = np.abs(jump) > 1e-2             # entries where s is well determined
    s = -2.0 * (F - 0.5 * (fl(QL) + fl(QR)))[ok] / jump[ok]
    face = np.broadcast_to(np.arange(5)[:, None, None], jump.shape)[ok]
    lam = np.maximum(pde.max_speed(np.moveaxis(QL, 1, 0), d), pde.max_speed(np.moveaxis(QR, 1, 0), d))
    for f in range(5):
        sf = s[face == f]
        assert len(sf) > 20
        assert np.allclose(sf, sf[0], rtol=1e-8)
        assert sf.min() >= lam[f].max() * (1 - 1e-8)
        assert sf.max() <= lam[f].max() * (1 + 1e-8)
    assert lam[2].max() > 1.5 * np.delete(lam[2], 4).max()


def test_cfl_rate_by_hand():
    """Uniform state: the rate is sum_d (|v_d| + c) / h_d, computed by hand."""
    pde = pdes.Euler(2)
    q = pde.primitive_to_conserved(1.0, [1.0, -2.0], 1.0 / 1.4)   # c = 1
    u = np.broadcast_to(q.reshape(1, 4, 1, 1), (3, 4, 2, 2)).copy()
    h = np.array([[0.5, 0.25]] * 3)
    assert abs(ader.cfl_rate(u, h, pde) - (2.0 / 0.5 + 3.0 / 0.25)) < 1e-12
    assert abs(ader.cfl_dt(u, h, pde, 3, cfl=0.5) - 0.5 / 16.0) < 1e-15
