"""Pins of the oracle's spacetree: balance, face coverage, skeleton, remesh."""
import itertools

import numpy as np
import pytest

from oracle import ader, basis, mesh as meshmod
from oracle_helpers import refined_mesh


def boxes(m):
    out = []
    for k in m.cells:
        h = m.width(k[0])
        a = m.lo + np.asarray(k[1], dtype=np.float64) * h
        out.append((a, a + h))
    return out


def touching_levels_bruteforce(m):
    """For every cell, the levels of all leaves that share a (d-1)-dimensional
    piece of face with it, found by box geometry with periodic shifts
    (vectorised over the other cells)."""
    bx = boxes(m)
    A = np.array([a for a, _ in bx])
    Bb = np.array([b for _, b in bx])
    lv = np.array([k[0] for k in m.cells])
    L = m.hi - m.lo
    res = []
    tol = 1e-12
    for i in range(len(bx)):
        a, b = A[i], Bb[i]
        found = set()
        for shift in itertools.product((-1, 0, 1), repeat=m.dim):
            sh = np.asarray(shift) * L
            c2, d2 = A + sh, Bb + sh
            touch = (np.abs(b - c2) < tol) | (np.abs(d2 - a) < tol)
            overlap = (np.minimum(b, d2) - np.maximum(a, c2)) > tol
            ok = (touch.sum(axis=1) == 1) & ((overlap & ~touch).sum(axis=1) == m.dim - 1)
            found.update(lv[ok].tolist())
        res.append(found)
    return res


@pytest.mark.parametrize("dim,base", [(2, 3), (2, 9), (3, 3)])
def test_uniform_faces(dim, base):
    m = meshmod.Mesh(dim, (base,) * dim, 2)
    conf, parents = m.faces()
    assert len(conf) == dim * base ** dim and not parents
    assert not m.skeleton().any()


@pytest.mark.parametrize("dim,base,levels", [(2, 9, 2), (2, 3, 2), (3, 3, 1), (3, 3, 2)])
def test_refined_mesh_balance_coverage_skeleton(dim, base, levels):
    m = refined_mesh(dim, base, levels, (0.45,) * dim, 0.2)
    lv = np.array([k[0] for k in m.cells])
    assert lv.max() == levels and lv.min() == 0
    # leaves tile the domain
    vol = np.prod(m.cell_widths(), axis=1).sum()
    assert abs(vol - 1.0) < 1e-12
    # 2:1 balance by geometry, and the skeleton = cells touching another level
    touch = touching_levels_bruteforce(m)
    skel_geo = np.zeros(len(m.cells), dtype=bool)
    for i, k in enumerate(m.cells):
        assert all(abs(l - k[0]) <= 1 for l in touch[i])
        skel_geo[i] = any(l != k[0] for l in touch[i])
    assert np.array_equal(skel_geo, m.skeleton())
    # every face slot of every cell is covered exactly once
    conf, parents = m.faces()
    count = np.zeros((len(m.cells), dim, 2), dtype=int)
    for a, b, dr in conf:
        count[a, dr, 1] += 1
        count[b, dr, 0] += 1
    for c, dr, side, kids in parents:
        count[c, dr, side] += 1
        assert len(kids) == 3 ** (dim - 1)
        for f, _ in kids:
            count[f, dr, 1 - side] += 1
            assert m.cells[f][0] == m.cells[c][0] + 1
    assert np.all(count == 1)


def test_balance_cascade():
    """Refining a corner cell twice forces the neighbours of the level-2
    cells to level >= 1 (a balance cascade), never more."""
    m = meshmod.Mesh(2, (3, 3), 3)
    B = basis.Basis(1)
    u = np.zeros((9, 1, 2, 2))
    flags = np.zeros(9, dtype=np.int8)
    flags[m.index[(0, (1, 1))]] = 1
    u = m.remesh(u, flags, B)
    flags = np.array([1 if k == (1, (3, 3)) else 0 for k in m.cells], dtype=np.int8)
    u = m.remesh(u, flags, B)
    lv = {k: k[0] for k in m.cells}
    assert max(lv.values()) == 2
    for i, ls in enumerate(touching_levels_bruteforce(m)):
        assert all(abs(l - m.cells[i][0]) <= 1 for l in ls)
    # the level-2 cells sit in (1,(3,3)); its face neighbours at level 1 exist
    assert (1, (2, 3)) in m.leaves and (1, (3, 2)) in m.leaves


@pytest.mark.parametrize("dim", [2, 3])
def test_remesh_transfer_identities(dim):
    """Refine then coarsen is the identity on the polynomial data; both keep
    the integral of every variable (conservative transfer)."""
    N = 3
    B = basis.Basis(N)
    m = meshmod.Mesh(dim, (3,) * dim, 1)
    rng = np.random.default_rng(4)
    u0 = rng.standard_normal((len(m.cells), 2) + (B.n,) * dim)
    I0 = ader.cell_integral(u0, m.cell_widths(), B)
    flags = np.zeros(len(m.cells), dtype=np.int8)
    flags[[0, 4]] = 1
    u1 = m.remesh(u0, flags, B)
    assert len(m.cells) == 3 ** dim - 2 + 2 * 3 ** dim
    assert np.allclose(ader.cell_integral(u1, m.cell_widths(), B), I0, atol=1e-13)
    flags = np.array([-1 if k[0] == 1 else 0 for k in m.cells], dtype=np.int8)
    u2 = m.remesh(u1, flags, B)
    assert len(m.cells) == 3 ** dim
    assert np.allclose(u2, u0, atol=1e-13)
    # coarsening of non-polynomial children: L2 projection keeps integrals
    m.remesh(u2, np.array([1 if i == 2 else 0 for i in range(len(m.cells))]), B)
    u3 = rng.standard_normal((len(m.cells), 2) + (B.n,) * dim)
    I3 = ader.cell_integral(u3, m.cell_widths(), B)
    flags = np.array([-1 if k[0] == 1 else 0 for k in m.cells], dtype=np.int8)
    u4 = m.remesh(u3, flags, B)
    assert np.allclose(ader.cell_integral(u4, m.cell_widths(), B), I3, atol=1e-13)


def test_coarsen_blocked_by_balance():
    """A family may not coarsen while a leaf two levels finer than the parent
    touches the parent's faces."""
    m = meshmod.Mesh(2, (3, 3), 3)
    B = basis.Basis(1)
    u = np.zeros((9, 1, 2, 2))
    u = m.remesh(u, [1 if k == (0, (1, 1)) else 0 for k in m.cells], B)
    u = m.remesh(u, [1 if k == (1, (3, 4)) else 0 for k in m.cells], B)   # left child column
    # ask every level-1 cell in parent (0,(1,1)) to coarsen: blocked? the
    # level-2 cells are inside that family, so (1,(3,4)) is not a leaf -> no
    fl = [-1 if k[0] == 1 and k[1][0] // 3 == 1 and k[1][1] // 3 == 1 else 0 for k in m.cells]
    n_before = len(m.cells)
    u = m.remesh(u, fl, B)
    assert len(m.cells) == n_before


def test_coarsen_blocked_by_finer_neighbour():
    """A complete family of flagged leaves stays refined while a leaf two
    levels finer than its parent touches one of the parent's faces: cell
    (0,(1,1)) is refined, and the level-1 cell left of it, (1,(2,4)), is
    refined again, so its level-2 children touch the family; coarsening the
    family would put level 0 next to level 2."""
    m = meshmod.Mesh(2, (3, 3), 3)
    B = basis.Basis(1)
    u = np.zeros((9, 1, 2, 2))
    u = m.remesh(u, [1 if k in ((0, (1, 1)), (0, (0, 1))) else 0 for k in m.cells], B)
    u = m.remesh(u, [1 if k == (1, (2, 4)) else 0 for k in m.cells], B)
    assert (2, (8, 13)) in m.leaves and (1, (3, 4)) in m.leaves
    family = [k for k in m.cells if k[0] == 1 and k[1][0] // 3 == 1 and k[1][1] // 3 == 1]
    assert len(family) == 9
    before = sorted(m.cells)
    u = m.remesh(u, [-1 if k in family else 0 for k in m.cells], B)
    assert sorted(m.cells) == before
    # and once the finer cells are gone, the same family coarsens
    u = m.remesh(u, [-1 if k[0] == 2 else 0 for k in m.cells], B)
    u = m.remesh(u, [-1 if k in family else 0 for k in m.cells], B)
    assert (0, (1, 1)) in m.leaves


@pytest.mark.parametrize("dim", [2, 3])
def test_prolong_face_equals_extrapolated_prolong_volume(dim):
    """Face-only prolongation (virtual-cell faces) equals extrapolating the
    volume interpolation of the coarse cell into the virtual cell."""
    N = 4
    B = basis.Basis(N)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 3) + (B.n,) * dim)
    for dr in range(dim):
        for side in range(2):
            face = ader.face_values(x, dr, side, B)
            for s in meshmod.subface_indices(dim, dr):
                full = []
                t = 0
                for a in range(dim):
                    if a == dr:
                        full.append(0 if side == 0 else 2)
                    else:
                        full.append(s[t])
                        t += 1
                vol = ader.prolong_volume(x, tuple(full), B)
                ref = ader.face_values(vol, dr, side, B)
                assert np.allclose(ader.prolong_face(face, s, B, dim), ref, atol=1e-13)


def test_gradient_indicator_of_linear_and_quadratic_fields():
    """eta = h |grad q| is exact for a linear field and for x^2 at the node of
    largest x (polynomials of degree <= N are differentiated exactly)."""
    from oracle import criterion
    N = 3
    B = basis.Basis(N)
    m = meshmod.Mesh(2, (3, 3), 1)
    X = m.node_coords(B.xi)
    u = np.stack([3.0 * X[0] - 4.0 * X[1], X[0] ** 2], axis=1)
    h = m.cell_widths()
    eta = criterion.gradient_indicator(u, h, B, 0)
    assert np.allclose(eta, 5.0 * h[:, 0], rtol=1e-12)
    eta2 = criterion.gradient_indicator(u, h, B, 1)
    xmax = (X[0].reshape(len(m.cells), -1)).max(axis=1)
    assert np.allclose(eta2, 2.0 * xmax * h[:, 0], rtol=1e-12)
    _, fl = criterion.gradient_flags(m, u, B, 0, 5.0 / 4, 5.0 / 10)
    assert fl.tolist() == [1 if 5.0 * hh > 5.0 / 4 else (-1 if k[0] > 0 and 5.0 * hh < 0.5 else 0)
                           for hh, k in zip(h[:, 0], m.cells)]


def test_gradient_indicator_anisotropic_cells():
    """On cells with h_x = 3 h_y the weight is the larger width:
    eta = h_max |grad q| = 5 h_x for q = 3x - 4y."""
    from oracle import criterion
    B = basis.Basis(2)
    m = meshmod.Mesh(2, (3, 9), 0)
    X = m.node_coords(B.xi)
    u = (3.0 * X[0] - 4.0 * X[1])[:, np.newaxis]
    h = m.cell_widths()
    assert np.allclose(h[:, 0], 3.0 * h[:, 1])
    assert np.allclose(criterion.gradient_indicator(u, h, B, 0), 5.0 * h[:, 0], rtol=1e-12)


def test_sphere_flags_periodic_distance_and_coarsening_rule():
    """The ball is measured with the periodic distance (a ball at x = 0.02
    reaches the last column of cells), and a leaf coarsens only when its
    parent's box misses the ball (a sibling of a cell that meets it stays)."""
    m = meshmod.Mesh(2, (9, 9), 1)
    fl = meshmod.sphere_flags(m, (0.02, 0.5), 0.05)
    assert fl[m.index[(0, (8, 4))]] == 1 and fl[m.index[(0, (0, 4))]] == 1
    assert fl[m.index[(0, (7, 4))]] == 0
    B = basis.Basis(1)
    m.remesh(np.zeros((81, 1, 2, 2)), fl, B)
    # the ball now moves so that it meets only the left column of the family of (0, (0, 4))
    fl = meshmod.sphere_flags(m, (0.0, 0.5), 0.02)
    sib = m.index[(1, (2, 13))]           # right column of that family: its own box misses the ball
    assert fl[sib] == 0
    gone = meshmod.sphere_flags(m, (0.5, 0.9), 0.02)
    assert gone[sib] == -1


def test_hessian_indicator_closed_forms():
    """eta = h^2 |H q|_F against closed forms on an anisotropic 2-level mesh
    (h_x != h_y, so a derivative taken along the wrong axis or divided by the
    wrong width fails): linear -> 0, y^2 -> 2 h^2, x y -> sqrt(2) h^2 (the mixed
    entries count), x^3 -> 6 max|x| h^2 (exact at N = 3), and in 3D
    x^2 + y^2 + z^2 -> 2 sqrt(3) h^2."""
    from oracle import criterion
    N = 3
    B = basis.Basis(N)
    m = meshmod.Mesh(2, (3, 9), 1)
    m.remesh(np.zeros((len(m.cells), 1) + (2, 2)), np.array([1] + [0] * (len(m.cells) - 1), dtype=np.int8),
             basis.Basis(1))
    X = m.node_coords(B.xi)
    h = m.cell_widths()
    assert not np.allclose(h[:, 0], h[:, 1])
    hm = h.max(axis=1)
    fields = [2.0 * X[0] - 5.0 * X[1] + 1.0, X[1] ** 2, X[0] * X[1], X[0] ** 3]
    u = np.stack(fields, axis=1)
    eta = [criterion.gradient_indicator(u, h, B, v, deriv=2) for v in range(4)]
    assert np.all(np.abs(eta[0]) < 1e-9 * hm ** 2 / h.min(axis=1) ** 2)
    assert np.allclose(eta[1], 2.0 * hm ** 2, rtol=1e-11)
    assert np.allclose(eta[2], np.sqrt(2.0) * hm ** 2, rtol=1e-11)
    xmax = np.abs(X[0].reshape(len(m.cells), -1)).max(axis=1)
    assert np.allclose(eta[3], 6.0 * xmax * hm ** 2, rtol=1e-11)
    m3 = meshmod.Mesh(3, (3, 3, 3), 0)
    X3 = m3.node_coords(B.xi)
    h3 = m3.cell_widths()
    u3 = np.stack([X3[0] ** 2 + X3[1] ** 2 + X3[2] ** 2], axis=1)
    eta3 = criterion.gradient_indicator(u3, h3, B, 0, deriv=2)
    assert np.allclose(eta3, 2.0 * np.sqrt(3.0) * h3.max(axis=1) ** 2, rtol=1e-11)
    thr = 2.0 / 81.0 * 1.0001      # between the fine cells' 2 (1/9)^2 and the coarse ones' 2 (1/3)^2
    _, fl = criterion.gradient_flags(m, u, B, 1, thr, thr, deriv=2)
    assert fl.tolist() == [1 if k[0] == 0 else -1 for k in m.cells]
