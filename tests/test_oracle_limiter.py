"""Pins of the oracle's a posteriori subcell FV limiter: the subcell operators
against closed forms, the all-limited step against an independent fine-grid
finite-volume step, conservation and free stream with limited and unlimited
cells side by side, and the detection rules."""
import numpy as np
import pytest

from oracle import ader, basis, limiter as lim, mesh as meshmod, pde as pdes
from oracle_helpers import refined_mesh, random_state
import workloads


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_subcell_averages_of_monomials(N):
    """A maps nodal values of x^k (k <= N) to its exact averages over the
    2N+1 subintervals: ((b^(k+1) - a^(k+1)) / (k+1)) / (b - a)."""
    B = basis.Basis(N)
    sc = lim.Subcells(B)
    S = 2 * N + 1
    a = np.arange(S) / S
    b = (np.arange(S) + 1) / S
    for k in range(N + 1):
        exact = (b ** (k + 1) - a ** (k + 1)) / ((k + 1) * (b - a))
        assert np.abs(sc.A @ B.xi ** k - exact).max() < 1e-14


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_reconstruction_inverts_and_conserves(N):
    B = basis.Basis(N)
    sc = lim.Subcells(B)
    assert np.abs(sc.R @ sc.A - np.eye(B.n)).max() < 1e-12
    # a degree-N polynomial is recovered from its exact subcell averages
    S = 2 * N + 1
    a, b = np.arange(S) / S, (np.arange(S) + 1) / S
    coef = np.random.default_rng(N).standard_normal(N + 1)
    avg = sum(c * (b ** (k + 1) - a ** (k + 1)) / ((k + 1) * (b - a)) for k, c in enumerate(coef))
    vals = sum(c * B.xi ** k for k, c in enumerate(coef))
    assert np.abs(sc.R @ avg - vals).max() < 1e-11
    # the cell mean of R v equals the mean of arbitrary averages v
    v = np.random.default_rng(10 + N).standard_normal(S)
    assert abs(B.w @ (sc.R @ v) - v.mean()) < 1e-14


@pytest.mark.parametrize("N,dim", [(2, 2), (3, 3), (5, 2)])
def test_face_projection_conserves(N, dim):
    """The projected face flux carries the same total as the subface fluxes,
    and a constant stays constant."""
    B = basis.Basis(N)
    sc = lim.Subcells(B)
    S = sc.S
    G = np.random.default_rng(N).standard_normal((3, S ** (dim - 1)))
    F = lim.project_face(G, sc, dim)
    W = B.w if dim == 2 else np.multiply.outer(B.w, B.w).ravel()
    assert np.allclose(F @ W, G.mean(axis=1), atol=1e-14, rtol=0)
    c = lim.project_face(np.full((1, S ** (dim - 1)), 2.5), sc, dim)
    assert np.abs(c - 2.5).max() < 1e-13


# ---------------------------------------------------------------- fine grid

def _euler_flux(q, d, gamma):
    rho = q[0]
    vel = [q[1 + a] / rho for a in range(len(q) - 2)]
    p = (gamma - 1.0) * (q[-1] - 0.5 * rho * sum(v * v for v in vel))
    f = [rho * vel[d]] + [rho * vel[a] * vel[d] + (p if a == d else 0.0)
                          for a in range(len(vel))] + [vel[d] * (q[-1] + p)]
    lam = np.abs(vel[d]) + np.sqrt(gamma * p / rho)
    return np.stack(f), lam


def _fine_grid_fv(V, dt, hs, gamma):
    """First-order Rusanov FV step on a periodic grid V[var, (z,) y, x],
    written with np.roll, independent of the oracle's patch code."""
    dim = V.ndim - 1
    out = V.copy()
    for d in range(dim):
        ax = V.ndim - 1 - d
        Vr = np.roll(V, -1, axis=ax)                 # right neighbour
        fL, lL = _euler_flux(V, d, gamma)
        fR, lR = _euler_flux(Vr, d, gamma)
        F = 0.5 * (fL + fR) - 0.5 * np.maximum(lL, lR) * (Vr - V)   # at i + 1/2
        out -= dt / hs[d] * (F - np.roll(F, 1, axis=ax))
    return out


def _to_global(v, m, S):
    dim = m.dim
    X = [b * S for b in m.base]
    V = np.zeros((v.shape[1],) + tuple(reversed(X)))
    for c, (lvl, x) in enumerate(m.cells):
        sl = tuple(slice(x[a] * S, (x[a] + 1) * S) for a in reversed(range(dim)))
        V[(slice(None),) + sl] = v[c]
    return V


def _from_global(V, m, S):
    out = []
    for lvl, x in m.cells:
        sl = tuple(slice(x[a] * S, (x[a] + 1) * S) for a in reversed(range(m.dim)))
        out.append(V[(slice(None),) + sl])
    return np.stack(out)


@pytest.mark.parametrize("dim,base,N", [(2, 4, 3), (2, 3, 2), (3, 2, 2)])
def test_all_limited_is_fine_grid_fv(dim, base, N):
    """Every cell limited on a uniform periodic mesh: the step is a plain FV
    step on the (2N+1)-times finer grid, read back to nodes by least squares;
    the next dt comes from the nodes and subcell averages of that state."""
    m = meshmod.Mesh(dim, (base,) * dim, 0)
    B = basis.Basis(N)
    P = pdes.Euler(dim)
    u = random_state(m, B, "euler", seed=5 + dim)
    h = m.cell_widths()
    dt = ader.cfl_dt(u, h, P, N)
    out = lim.step_limited(m, u, dt, P, B, force=np.ones(len(m.cells), bool))
    assert out.limited.all() and not out.kept.any() and not out.fixed.any()
    sc = lim.Subcells(B)
    S = sc.S
    V = _to_global(lim.averages(u, sc), m, S)
    Vn = _fine_grid_fv(V, dt, h[0] / S, P.gamma)
    v_new = _from_global(Vn, m, S)
    assert np.abs(out.u - lim.to_nodes(v_new, sc)).max() < 1e-12
    rate_nodes = ader.cfl_rate(out.u, h, P)
    rate_sub = ader.cfl_rate(v_new, h, P)
    from oracle.stability import cfl_number
    assert abs(out.dt_next - cfl_number(N) / max(rate_nodes, rate_sub)) < 1e-15 * out.dt_next


# ------------------------------------------------------- mixed DG/FV steps

@pytest.mark.parametrize("dim,base,N,pde_name", [(2, 5, 3, "euler"), (3, 3, 2, "euler"),
                                                  (2, 5, 2, "acoustics")])
def test_mixed_step_conserves(dim, base, N, pde_name):
    """Limited and unlimited cells side by side on a periodic mesh: the
    integral of every variable is unchanged (the unlimited neighbours lift
    the projected FV fluxes)."""
    m = meshmod.Mesh(dim, (base,) * dim, 0)
    B = basis.Basis(N)
    P = pdes.make_pde(pde_name, dim)
    u = random_state(m, B, pde_name, seed=31)
    h = m.cell_widths()
    dt = ader.cfl_dt(u, h, P, N)
    force = np.random.default_rng(3).random(len(m.cells)) < 0.3
    out = lim.step_limited(m, u, dt, P, B, force=force)
    assert out.limited.sum() >= force.sum() and out.fixed.any()
    I0 = ader.cell_integral(u, h, B)
    I1 = ader.cell_integral(out.u, h, B)
    assert np.allclose(I1, I0, atol=1e-13, rtol=0), I1 - I0
    # without the flux replacement the mixed step would not conserve
    naive = out.candidate.u.copy()
    naive[out.limited] = out.u[out.limited]
    assert np.abs(ader.cell_integral(naive, h, B) - I0).max() > 1e-9


def test_mixed_step_free_stream():
    m = meshmod.Mesh(2, (5, 5), 0)
    B = basis.Basis(3)
    P = pdes.Euler(2)
    q0 = P.primitive_to_conserved(1.2, [0.7, -0.3], 0.8)
    u = np.broadcast_to(q0.reshape(1, -1, 1, 1), (25, 4, 4, 4)).copy()
    force = np.zeros(25, bool)
    force[[0, 7, 12, 13]] = True
    out = lim.step_limited(m, u, 0.01, P, B, force=force)
    assert np.abs(out.u - u).max() < 1e-14


# ------------------------------------------------------------- detection

def _uniform(dim, base, N, value):
    m = meshmod.Mesh(dim, (base,) * dim, 0)
    B = basis.Basis(N)
    u = np.broadcast_to(np.asarray(value).reshape((1, -1) + (1,) * dim),
                        (len(m.cells), len(value)) + (B.n,) * dim).copy()
    return m, B, u


def test_detection_rules():
    P = pdes.Euler(2)
    q0 = P.primitive_to_conserved(1.0, [0.2, 0.1], 1.0)
    m, B, u = _uniform(2, 4, 3, q0)
    sc, nb = lim.Subcells(B), lim.neighbors(m)
    lmt, kept = lim.detect(P, u, u.copy(), sc, nb)
    assert not lmt.any() and not kept.any()
    # a constant shift of one cell's energy: within delta0 = 1e-4 -> accepted,
    # beyond it -> troubled (the neighbourhood has max - min = 0)
    for shift, want in ((0.9e-4, False), (1.1e-4, True)):
        cand = u.copy()
        cand[5, 3] += shift
        lmt, _ = lim.detect(P, u, cand, sc, nb)
        assert lmt[5] == want and lmt.sum() == int(want)
    # the relative part: delta = 1e-3 (max - min) over the cell and its face
    # neighbours; a neighbour raised by 1 makes delta = 1e-3
    old = u.copy()
    old[6, 0] += 1.0                  # cell 6 shares a face with cell 5
    cand = old.copy()
    cand[5, 0] = old[5, 0] - 0.9e-3
    assert not lim.detect(P, old, cand, sc, nb)[0][5]
    cand[5, 0] = old[5, 0] - 1.1e-3
    assert lim.detect(P, old, cand, sc, nb)[0][5]
    # negative pressure at one node, non-finite value
    cand = u.copy()
    cand[2, 3, 1, 1] = 0.0
    assert lim.detect(P, u, cand, sc, nb)[0][2]
    cand = u.copy()
    cand[9, 1, 0, 0] = np.nan
    lmt, _ = lim.detect(P, u, cand, sc, nb)
    assert lmt[9] and lmt.sum() == 1


def test_detection_admissibility_alone():
    """With the candidate equal to u(T) the maximum principle holds trivially,
    so only admissibility can flag: a node with rho > 0 but p < 0, and a cell
    whose nodal densities are all positive while the polynomial's average over
    an edge subcell is negative."""
    P = pdes.Euler(2)
    q0 = P.primitive_to_conserved(1.0, [0.0, 0.0], 1.0)
    m, B, u = _uniform(2, 4, 3, q0)
    sc, nb = lim.Subcells(B), lim.neighbors(m)
    cand = u.copy()
    cand[3, 1, 2, 1] = 3.0                 # rho v_x = 3 at one node: kinetic energy 4.5 > E = 2.5
    assert P.pressure(cand[3, :, 2, 1]) < 0 < cand[3, 0, 2, 1]
    lmt, _ = lim.detect(P, cand, cand, sc, nb)
    assert lmt[3] and lmt.sum() == 1
    cand = u.copy()
    eps = 1e-3
    cand[7, 0] = np.array([1.0, eps, eps, 1.0])[np.newaxis, :]   # rho along x, at rest: p stays 1
    v = lim.averages(cand[7:8], sc)[0, 0]
    assert (cand[7, 0] > 0).all() and v.min() < 0
    lmt, _ = lim.detect(P, cand, cand, sc, nb)
    assert lmt[7] and lmt.sum() == 1


def test_detection_bounds_include_the_neighbours():
    """The relaxed maximum principle takes its bounds over the cell and its
    face neighbours: a candidate that leaves its own cell's range but stays
    inside a neighbour's is accepted, in both directions."""
    P = pdes.Euler(2)
    q0 = P.primitive_to_conserved(1.0, [0.2, 0.1], 1.0)
    m, B, u = _uniform(2, 4, 3, q0)
    sc, nb = lim.Subcells(B), lim.neighbors(m)
    for sign in (-1.0, 1.0):
        old = u.copy()
        old[6, 0] += sign * 0.5            # cell 6 shares a face with cell 5
        cand = old.copy()
        cand[5, 0] += sign * 0.3
        assert not lim.detect(P, old, cand, sc, nb)[0][5]
        cand[5, 0] = old[5, 0] + sign * 0.6
        assert lim.detect(P, old, cand, sc, nb)[0][5]


def test_no_limiting_across_transitions():
    """A forced cell with a non-conforming face keeps its DG candidate."""
    m = refined_mesh(2, 9, 1, (0.5, 0.5), 0.1)
    B = basis.Basis(2)
    P = pdes.Euler(2)
    u = random_state(m, B, "euler", seed=4)
    nb = lim.neighbors(m)
    at_transition = ~(nb >= 0).all(axis=(1, 2))
    assert at_transition.any()
    force = np.zeros(len(m.cells), bool)
    c_tr = int(np.flatnonzero(at_transition)[0])
    c_in = int(np.flatnonzero(~at_transition & (m.cell_widths()[:, 0] > 0.1))[0])
    force[[c_tr, c_in]] = True
    dt = ader.cfl_dt(u, m.cell_widths(), P, 2)
    out = lim.step_limited(m, u, dt, P, B, force=force)
    assert out.kept[c_tr] and not out.limited[c_tr]
    assert out.limited[c_in]
    assert np.array_equal(out.u[c_tr], out.candidate.u[c_tr])
    h = m.cell_widths()
    assert np.allclose(ader.cell_integral(out.u, h, B), ader.cell_integral(u, h, B),
                       atol=1e-13, rtol=0)


def test_explosion_limits_near_the_shock():
    """Circular explosion (a density and pressure jump): the limiter flags
    cells along the discontinuity only and keeps the state admissible."""
    m = meshmod.Mesh(2, (27, 27), 0)
    B = basis.Basis(3)
    P = pdes.Euler(2)
    X = m.node_coords(B.xi)
    q = workloads.circular_explosion(X, width=0.02)
    u = np.ascontiguousarray(np.moveaxis(q, 0, 1))
    h = m.cell_widths()
    dt = ader.cfl_dt(u, h, P, 3)
    c = np.stack([(np.asarray(k[1]) + 0.5) / 27 for k in m.cells])
    r = np.sqrt(((c - 0.5) ** 2).sum(axis=1))
    for _ in range(3):
        out = lim.step_limited(m, u, dt, P, B)
        assert 0 < out.limited.sum() < len(m.cells) // 2
        assert np.abs(r[out.limited] - workloads.EXPLOSION_RADIUS).max() < 4.0 / 27
        assert np.isfinite(out.u).all() and (out.u[:, 0] > 0).all()
        assert (P.pressure(np.moveaxis(out.u, 1, 0)) > 0).all()
        u, dt = out.u, out.dt_next


def test_refine_flags_around_troubled_cells():
    """Troubled cells and their face neighbours (across transitions too) are
    refined below the finest level; every other cell above level 0 coarsens."""
    m = refined_mesh(2, 9, 2, (0.5, 0.5), 0.1, rounds=1)
    troubled = np.zeros(len(m.cells), dtype=bool)
    levels = np.array([k[0] for k in m.cells])
    c0 = int(np.flatnonzero(levels == 1)[0])
    c1 = int(np.flatnonzero(levels == 0)[0])
    troubled[[c0, c1]] = True
    flags = lim.refine_flags(m, troubled)
    nb = lim.face_neighbours(m)
    marked = set([c0, c1]) | nb[c0] | nb[c1]
    for i, (lvl, _) in enumerate(m.cells):
        if i in marked:
            assert flags[i] == (1 if lvl < m.max_level else 0)
        else:
            assert flags[i] == (-1 if lvl > 0 else 0)
    # a level-1 cell at the transition has its coarse neighbour among its face neighbours
    trans = [i for i in range(len(m.cells)) if levels[i] == 1 and any(levels[j] == 0 for j in nb[i])]
    assert trans
    # symmetric neighbour relation, 2d faces per cell at least
    for i in range(len(m.cells)):
        assert all(i in nb[j] for j in nb[i]) and len(nb[i]) >= 4


def test_refine_flags_at_the_finest_level():
    """A troubled cell already at the finest level keeps its level (flag 0),
    like its finest-level neighbours; a coarser troubled neighbourhood refines."""
    m = refined_mesh(2, 9, 2, (0.5, 0.5), 0.1)
    levels = np.array([k[0] for k in m.cells])
    fine = int(np.flatnonzero(levels == m.max_level)[0])
    troubled = np.zeros(len(m.cells), dtype=bool)
    troubled[fine] = True
    flags = lim.refine_flags(m, troubled)
    assert flags[fine] == 0
    nb = lim.face_neighbours(m)
    for j in nb[fine]:
        assert flags[j] == (1 if levels[j] < m.max_level else 0)
