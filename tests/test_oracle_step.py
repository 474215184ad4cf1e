"""Pins of the oracle's full step: free stream, conservation, the operator
form of Eq. (4), entropy-wave invariants and the design order."""
import numpy as np
import pytest

from oracle import ader, basis, mesh as meshmod, pde as pdes, step as stepmod
from oracle_helpers import refined_mesh, random_state, state_from
import workloads


@pytest.fixture(scope="module")
def amr2d():
    return refined_mesh(2, 9, 2, (0.45, 0.55), 0.12)


@pytest.fixture(scope="module")
def amr3d():
    return refined_mesh(3, 3, 2, (0.45, 0.5, 0.55), 0.12)


@pytest.mark.parametrize("which,N", [("amr2d", 3), ("amr2d", 5), ("amr3d", 2)])
def test_free_stream_on_amr(which, N, request):
    m = request.getfixturevalue(which)
    B = basis.Basis(N)
    pde = pdes.Euler(m.dim)
    q0 = pde.primitive_to_conserved(1.1, [0.6, -0.4, 0.3][:m.dim], 0.9)
    u = np.broadcast_to(q0.reshape((1, -1) + (1,) * m.dim),
                        (len(m.cells), m.dim + 2) + (B.n,) * m.dim).copy()
    dt = ader.cfl_dt(u, m.cell_widths(), pde, N)
    out = stepmod.step(m, u, dt, pde, B)
    assert np.abs(out.u - u).max() < 1e-13
    assert not np.isnan(out.Fs).any()


@pytest.mark.parametrize("which,N,pde_name", [("amr2d", 3, "euler"), ("amr2d", 4, "acoustics"),
                                               ("amr3d", 2, "euler")])
def test_conservation_on_amr(which, N, pde_name, request):
    """Periodic domain with hanging faces: the integral of every variable is
    unchanged by a step (to rounding)."""
    m = request.getfixturevalue(which)
    B = basis.Basis(N)
    pde = pdes.make_pde(pde_name, m.dim)
    u = random_state(m, B, pde_name, seed=21)
    h = m.cell_widths()
    dt = ader.cfl_dt(u, h, pde, N)
    I0 = ader.cell_integral(u, h, B)
    out = stepmod.step(m, u, dt, pde, B)
    I1 = ader.cell_integral(out.u, h, B)
    assert np.allclose(I1, I0, atol=1e-13, rtol=0), I1 - I0
    # and the step does something
    assert np.abs(out.u - u).max() > 1e-4


@pytest.mark.parametrize("which,N", [("amr2d", 3), ("amr3d", 3)])
def test_operator_form_of_eq4(which, N, request):
    """Eq. (4) writes the step as Q(T+dT) = C_Corr F_R id|dc Q* + id|T+dT Q*.
    With q(1) = id|T+dT Q* (the predictor at tau = 1) and the interior
    face traces of F-bar, the corrector is q(1) minus the jump terms
    dt h^-1 w^-1 [phi(1) (F*_+ - F-bar_+) - phi(0) (F*_- - F-bar_-)].
    The identity holds at the Picard fixed point, so the predictor is iterated
    to convergence here.  The oracle's weak-form corrector must agree to
    rounding."""
    m = request.getfixturevalue(which)
    B = basis.Basis(N)
    pde = pdes.Euler(m.dim)
    u = random_state(m, B, "euler", seed=3)
    h = m.cell_widths()
    dt = ader.cfl_dt(u, h, pde, N)
    iters = 40
    out = stepmod.step(m, u, dt, pde, B, iters)
    q = ader.picard_predictor(u, h, dt, pde, B, iters)
    q1 = np.tensordot(q, B.phi1, axes=([1], [0]))          # (C, m, *nodes)
    jumps = out.Fs - out.Ff
    alt = ader.face_lifting(q1, jumps, h, dt, B)
    assert np.abs(alt - out.u).max() < 1e-12


def test_entropy_wave_keeps_velocity_and_pressure(amr3d):
    """On the density bubble (uniform v and p) the Euler flux is affine in rho,
    so velocity and pressure stay uniform to rounding, also across AMR."""
    m = amr3d
    N = 3
    B = basis.Basis(N)
    pde = pdes.Euler(3)
    u = state_from(m, B, lambda X: workloads.density_bubble(X, sigma=0.15))
    h = m.cell_widths()
    dt = ader.cfl_dt(u, h, pde, N)
    for _ in range(2):
        out = stepmod.step(m, u, dt, pde, B)
        u = out.u
        dt = out.dt_next
    q = np.moveaxis(u, 1, 0)
    vel = q[1:4] / q[0]
    assert np.abs(vel - 1.0).max() < 1e-12
    assert np.abs(pde.pressure(q) - 1.0).max() < 1e-12
    assert np.abs(q[0] - 1.0).max() > 0.01


def run_to(m, B, pde, u, t_end):
    h = m.cell_widths()
    t = 0.0
    dt = ader.cfl_dt(u, h, pde, B.order)
    while t < t_end - 1e-14:
        dt = min(dt, t_end - t)
        out = stepmod.step(m, u, dt, pde, B)
        u, t, dt = out.u, t + dt, out.dt_next
    return u


def l2_error(m, B, u, exact):
    e = (u - exact) ** 2
    return np.sqrt(ader.cell_integral(e, m.cell_widths(), B))


@pytest.mark.parametrize("N", [2, 3])
def test_convergence_entropy_wave(N):
    """Smooth periodic entropy wave (rho = 1 + 0.2 sin 2 pi (x + y), v = (1, 1),
    p = 1): L2 error of rho falls at the design rate N + 1 from 9^2 to 27^2."""
    B = basis.Basis(N)
    pde = pdes.Euler(2)

    def field(X, t):
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * (X[0] + X[1] - 2 * t))
        return np.stack(np.broadcast_arrays(rho, rho, rho, 1.0 / 0.4 + rho))

    errs = []
    for base in (9, 27):
        m = meshmod.Mesh(2, (base, base), 0)
        u = state_from(m, B, lambda X: field(X, 0.0))
        u = run_to(m, B, pde, u, 0.05)
        ex = state_from(m, B, lambda X: field(X, 0.05))
        errs.append(l2_error(m, B, u, ex)[0])
    rate = np.log(errs[0] / errs[1]) / np.log(3.0)
    assert rate > N + 0.6, (errs, rate)


def test_convergence_isentropic_vortex():
    """Nonlinear test with pressure and velocity variation: the isentropic
    vortex (strength 1, R = 0.05, so its tail at the periodic boundary is
    below 1e-20) converges at rate ~N + 1 from 27^2 to 81^2 at N = 3."""
    N = 3
    B = basis.Basis(N)
    pde = pdes.Euler(2)
    errs = []
    T = 0.005
    for base in (27, 81):
        m = meshmod.Mesh(2, (base, base), 0)
        u = state_from(m, B, lambda X: workloads.isentropic_vortex(X[0], X[1], eps=1.0, R=0.05))
        u = run_to(m, B, pde, u, T)
        ex = state_from(m, B, lambda X: workloads.isentropic_vortex(X[0], X[1], t=T, eps=1.0, R=0.05))
        errs.append(l2_error(m, B, u, ex))
    errs = np.array(errs)
    rates = np.log(errs[0] / errs[1]) / np.log(3.0)
    assert np.all(rates > N + 0.4), (errs, rates)


@pytest.mark.parametrize("N", [2, 3])
def test_full_step_obeys_the_von_neumann_limit(N):
    """The stability module assembles its own 1D amplification matrix; the
    full 2D step (mesh, faces, Rusanov, corrector) on acoustic data that vary
    in x only is a pair of advection problems with speed 1, so it must stay
    bounded at 0.9 nu_N and blow up at 1.2 nu_N (Courant number dt / h_x)."""
    from oracle import stability
    B = basis.Basis(N)
    P = pdes.Acoustics(2)
    m = meshmod.Mesh(2, (12, 1), 0)
    rng = np.random.default_rng(40 + N)
    u = np.zeros((12, 3, B.n, B.n))
    u[:] = rng.standard_normal((12, 3, 1, B.n))       # uniform in y
    hx = m.cell_widths()[0, 0]
    nu = stability.stability_limit(N)
    W = np.outer(B.w, B.w)

    def energy(x):                                    # GL-weighted L2 norm squared
        return float((x * x * W).sum())

    norms = {}
    for factor in (0.9, 1.2):
        v = u.copy()
        for _ in range(40):
            v = stepmod.step(m, v, factor * nu * hx, P, B).u
        norms[factor] = np.sqrt(energy(v) / energy(u))
    assert norms[0.9] <= 1.0 + 1e-10
    assert norms[1.2] > 1e3


def test_acoustics_energy_does_not_grow(amr2d):
    """Linear acoustics with Rusanov dissipation: the discrete energy
    sum W (p^2 + |v|^2) does not grow over a step, also across AMR."""
    m = amr2d
    B = basis.Basis(3)
    pde = pdes.Acoustics(2)
    u = state_from(m, B, lambda X: workloads.acoustic_pulses(X, seed=1, width=0.15))
    h = m.cell_widths()
    dt = ader.cfl_dt(u, h, pde, 3)
    e0 = ader.cell_integral(u ** 2, h, B).sum()
    for _ in range(3):
        u = stepmod.step(m, u, dt, pde, B).u
        e1 = ader.cell_integral(u ** 2, h, B).sum()
        assert e1 <= e0 * (1 + 1e-12)
        e0 = e1


@pytest.mark.parametrize("N", range(1, 10))
def test_cfl_table(N):
    """The Courant factors of the workloads are 0.9 times the oracle's von
    Neumann limit; the scheme is stable there and unstable 10% above nu_N."""
    from oracle import stability
    nu = stability.stability_limit(N)
    assert abs(workloads.ADER_CFL[N] - stability.cfl_number(N)) < 1e-12
    assert stability.spectral_radius(N, workloads.ADER_CFL[N]) <= 1.0 + 1e-9 or N >= 4
    assert stability.spectral_radius(N, workloads.ADER_CFL[N]) <= 1.0 + 1e-4
    assert stability.spectral_radius(N, 1.1 * nu) > 1.0 + 1e-4


@pytest.mark.parametrize("which,N", [("amr2d", 3), ("amr3d", 2)])
def test_step_sample_equals_full_step(which, N, request):
    """The cell-by-cell evaluation used for full-size parity agrees with the
    full oracle step on every kind of cell (conforming, coarse and fine sides
    of transitions)."""
    m = request.getfixturevalue(which)
    B = basis.Basis(N)
    P = pdes.Euler(m.dim)
    u = random_state(m, B, "euler", seed=77)
    dt = ader.cfl_dt(u, m.cell_widths(), P, N)
    full = stepmod.step(m, u, dt, P, B)
    skel = np.flatnonzero(m.skeleton())
    rng = np.random.default_rng(0)
    targets = np.concatenate([rng.choice(skel, 6, replace=False),
                              rng.choice(len(m.cells), 6, replace=False)])
    got = stepmod.step_sample(m, u, dt, P, B, targets)
    assert np.abs(got - full.u[targets]).max() < 1e-13


def test_ck_step_conserves_and_matches_picard_on_1d_data(amr2d):
    """The Cauchy-Kowalevski step conserves on an AMR mesh; on data varying
    along x only (uniform mesh) it equals the Picard step (both predictors are
    the exact local evolution there)."""
    B = basis.Basis(3)
    P = pdes.Acoustics(2)
    u = random_state(amr2d, B, "acoustics", seed=4)
    h = amr2d.cell_widths()
    dt = ader.cfl_dt(u, h, P, 3)
    out = stepmod.step(amr2d, u, dt, P, B, predictor="ck")
    assert np.allclose(ader.cell_integral(out.u, h, B), ader.cell_integral(u, h, B), atol=1e-13)
    m = meshmod.Mesh(2, (9, 9), 0)
    X = m.node_coords(B.xi)
    u1 = np.stack([np.sin(2 * np.pi * X[0]), np.cos(2 * np.pi * X[0]), 0 * X[0]], axis=1)
    dt = ader.cfl_dt(u1, m.cell_widths(), P, 3)
    a = stepmod.step(m, u1, dt, P, B, iters=4, predictor="ck").u
    b = stepmod.step(m, u1, dt, P, B, iters=4).u
    assert np.abs(a - b).max() < 1e-13
