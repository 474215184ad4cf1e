"""Adaptive 3^d spacetree mesh (oracle; test infrastructure).

Sec. 2.3 of the paper: a conformal base grid at level l_min, every refined cell
split into 3^d children (three-partitioning), the unrefined cells forming the
adaptive mesh.  Here a cell is the key (level, (i_x, i_y[, i_z])) with integer
coordinates in the grid of ``base * 3**level`` cells per axis; the domain is a
periodic box.  The tree is held as a set of leaves; a node is refined when it
has a leaf below it.

Faces (Sec. 2.3):

* a conforming face joins two leaves of one level;
* at a resolution transition the coarse cell's face is a parent face, split
  into 3^(d-1) child faces that coincide with faces of the finer leaves.
  Riemann solves run on the child faces only, on data prolonged from the
  coarse cell (virtual cells), and their results are restricted and
  accumulated into the parent face.

Child faces of a parent are enumerated in lexicographic order of the
sub-face index s (lowest tangential direction fastest); restriction sums them
in that order.

Remeshing (Sec. 2.3, the AMR epilogue of the corrector) takes one flag per
leaf (+1 refine, -1 coarsen, 0 keep) and applies, in this order:
  1. refine every flagged leaf below ``max_level``;
  2. 2:1 balance: refine any leaf with a face neighbour two or more levels
     finer, to a fixpoint (face balance only);
  3. coarsen a family of 3^d leaf siblings when all carry -1, are still leaves
     and no leaf across a face of the parent is two or more levels finer than
     the parent;
  4. transfer the solution: copy, interpolate into refined children, or
     L2-project coarsened children onto the parent.
"""
import itertools

import numpy as np

from .ader import prolong_volume, restrict_volume


def parent(key):
    lvl, x = key
    return (lvl - 1, tuple(c // 3 for c in x))


def children(key):
    lvl, x = key
    dim = len(x)
    out = []
    # lexicographic in (s_z, s_y, s_x) ... lowest direction fastest
    for s in itertools.product(range(3), repeat=dim):
        s = tuple(reversed(s))
        out.append(((lvl + 1, tuple(3 * x[a] + s[a] for a in range(dim))), s))
    return out


def subface_indices(dim, dr):
    """All sub-face indices s (tuple over tangential directions, lowest first),
    in lexicographic order with the lowest tangential direction fastest."""
    out = []
    for s in itertools.product(range(3), repeat=dim - 1):
        out.append(tuple(reversed(s)))
    return out


class Mesh:
    def __init__(self, dim, base, max_level, lo=None, hi=None):
        self.dim = dim
        self.base = tuple(base)
        self.max_level = max_level
        self.lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)
        self.hi = np.ones(dim) if hi is None else np.asarray(hi, dtype=np.float64)
        ranges = [range(b) for b in self.base]
        self.leaves = set((0, tuple(reversed(c))) for c in itertools.product(*reversed(ranges)))
        self._rebuild()

    # ----------------------------------------------------------------- tree
    def _rebuild(self):
        self.refined = set()
        for key in self.leaves:
            k = key
            while k[0] > 0:
                k = parent(k)
                if k in self.refined:
                    break
                self.refined.add(k)
        self.cells = sorted(self.leaves)
        self.index = {k: i for i, k in enumerate(self.cells)}

    def dims(self, level):
        return tuple(b * 3 ** level for b in self.base)

    def width(self, level):
        return (self.hi - self.lo) / np.asarray(self.dims(level), dtype=np.float64)

    def neighbor(self, key, dr, side):
        """Same-level node across the face (dr, side) (side 0: -dr, 1: +dr)."""
        lvl, x = key
        n = self.dims(lvl)[dr]
        y = list(x)
        y[dr] = (y[dr] + (1 if side == 1 else -1)) % n
        return (lvl, tuple(y))

    def exists(self, key):
        return key in self.leaves or key in self.refined

    def cell_widths(self):
        return np.stack([self.width(k[0]) for k in self.cells])

    def cell_origin(self, key):
        lvl, x = key
        return self.lo + np.asarray(x, dtype=np.float64) * self.width(lvl)

    def node_coords(self, xi):
        """Physical coordinates of all nodes: list over directions of arrays
        (C, *nodes) in the oracle's node layout."""
        C = len(self.cells)
        n = len(xi)
        out = []
        org = np.stack([self.cell_origin(k) for k in self.cells])
        h = self.cell_widths()
        for dr in range(self.dim):
            shape = [1] * self.dim
            shape[self.dim - 1 - dr] = n
            v = org[:, dr].reshape((C,) + (1,) * self.dim) + \
                h[:, dr].reshape((C,) + (1,) * self.dim) * np.asarray(xi).reshape(shape)
            out.append(np.broadcast_to(v, (C,) + (n,) * self.dim).copy())
        return out

    # ---------------------------------------------------------------- faces
    def touching_children(self, key, dr, side_of_key):
        """Children of node ``key`` that touch its face (dr, side_of_key), in
        sub-face order, as (child key, s)."""
        lvl, x = key
        out = []
        for s in subface_indices(self.dim, dr):
            loc = [0] * self.dim
            t = 0
            for a in range(self.dim):
                if a == dr:
                    loc[a] = 0 if side_of_key == 0 else 2
                else:
                    loc[a] = s[t]
                    t += 1
            out.append(((lvl + 1, tuple(3 * x[a] + loc[a] for a in range(self.dim))), s))
        return out

    def faces(self):
        """Conforming faces and parent faces of the current mesh.

        Returns ``(conf, parents)``:
          conf    - list of (left cell, right cell, dr)
          parents - list of (coarse cell, dr, coarse side, [(fine cell, s), ...])
        """
        conf, parents = [], []
        for key in self.cells:
            for dr in range(self.dim):
                nb = self.neighbor(key, dr, 1)
                if nb in self.leaves:
                    conf.append((self.index[key], self.index[nb], dr))
                elif nb in self.refined:
                    kids = self.touching_children(nb, dr, 0)
                    for ck, _ in kids:
                        assert ck in self.leaves, "mesh not 2:1 balanced"
                    parents.append((self.index[key], dr, 1,
                                    [(self.index[ck], s) for ck, s in kids]))
                nb = self.neighbor(key, dr, 0)
                if nb in self.refined:
                    kids = self.touching_children(nb, dr, 1)
                    for ck, _ in kids:
                        assert ck in self.leaves, "mesh not 2:1 balanced"
                    parents.append((self.index[key], dr, 0,
                                    [(self.index[ck], s) for ck, s in kids]))
        return conf, parents

    def max_level_across(self, key, dr, side):
        """Finest level of the leaves across face (dr, side) of node ``key``
        (a coarser leaf reports its own, lower, level)."""
        nb = self.neighbor(key, dr, side)
        if nb in self.leaves:
            return nb[0]
        if nb in self.refined:
            best = nb[0]
            for ck, _ in self.touching_children(nb, dr, 1 - side):
                best = max(best, self._max_level_below_face(ck, dr, 1 - side))
            return best
        return key[0] - 1

    def _max_level_below_face(self, key, dr, side):
        if key in self.leaves:
            return key[0]
        best = key[0]
        for ck, _ in self.touching_children(key, dr, side):
            best = max(best, self._max_level_below_face(ck, dr, side))
        return best

    def skeleton(self, refine_flags=None):
        """Boolean per cell: adjacent to a resolution transition (either side)
        or flagged for refinement (Sec. 3 and 3.1, skeleton cells)."""
        skel = np.zeros(len(self.cells), dtype=bool)
        _, parents = self.faces()
        for c, _, _, kids in parents:
            skel[c] = True
            for f, _ in kids:
                skel[f] = True
        if refine_flags is not None:
            skel |= np.asarray(refine_flags) > 0
        return skel

    # --------------------------------------------------------------- remesh
    def remesh(self, u, flags, B):
        """Apply refine/coarsen flags (one per leaf in ``self.cells`` order) and
        transfer the solution u[c, var, *nodes].  Returns the new u."""
        old_cells = list(self.cells)
        old_index = dict(self.index)
        flags = np.asarray(flags)
        coarsen = set(k for k, f in zip(old_cells, flags) if f < 0 and k[0] > 0)
        # 1. refine flagged leaves
        for k, f in zip(old_cells, flags):
            if f > 0 and k[0] < self.max_level:
                self._split(k)
        self._rebuild()
        # 2. 2:1 face balance to a fixpoint
        changed = True
        while changed:
            changed = False
            for k in list(self.cells):
                if k not in self.leaves:
                    continue
                for dr in range(self.dim):
                    for side in range(2):
                        if self.max_level_across(k, dr, side) >= k[0] + 2:
                            self._split(k)
                            changed = True
                            break
                    if k not in self.leaves:
                        break
            if changed:
                self._rebuild()
        # 3. coarsen complete families of flagged leaves
        fams = sorted(set(parent(k) for k in coarsen if k in self.leaves))
        approved = []
        for P in fams:
            kids = [ck for ck, _ in children(P)]
            if not all(ck in self.leaves and ck in coarsen for ck in kids):
                continue
            ok = True
            for dr in range(self.dim):
                for side in range(2):
                    if self.max_level_across(P, dr, side) >= P[0] + 2:
                        ok = False
            if ok:
                approved.append(P)
        for P in approved:
            for ck, _ in children(P):
                self.leaves.discard(ck)
            self.leaves.add(P)
        self._rebuild()
        # 4. transfer
        shape = (len(self.cells),) + u.shape[1:]
        unew = np.empty(shape)
        for i, k in enumerate(self.cells):
            if k in old_index:
                unew[i] = u[old_index[k]]
            elif k[0] > 0 and parent(k) in old_index:
                p = parent(k)
                s = tuple(k[1][a] - 3 * p[1][a] for a in range(self.dim))
                unew[i] = prolong_volume(u[old_index[p]][np.newaxis], s, B)[0]
            else:
                acc = np.zeros(u.shape[1:])
                for ck, s in children(k):
                    acc += restrict_volume(u[old_index[ck]][np.newaxis], s, B)[0]
                unew[i] = acc
        return unew

    def _split(self, key):
        self.leaves.discard(key)
        for ck, _ in children(key):
            self.leaves.add(ck)


def sphere_flags(mesh, center, radius):
    """Geometric criterion: refine a leaf below ``max_level`` whose box meets
    the ball B(center, radius) (periodic distance); coarsen a leaf above level
    0 whose parent's box misses the ball."""
    L = mesh.hi - mesh.lo
    center = np.asarray(center, dtype=np.float64)

    def meets(key):
        lvl, x = key
        h = mesh.width(lvl)
        a = mesh.lo + np.asarray(x, dtype=np.float64) * h
        b = a + h
        dist2 = 0.0
        for dr in range(mesh.dim):
            best = None
            for shift in (-L[dr], 0.0, L[dr]):
                c = center[dr] + shift
                g = max(a[dr] - c, 0.0, c - b[dr])
                best = g if best is None else min(best, g)
            dist2 += best * best
        return dist2 <= radius * radius

    flags = np.zeros(len(mesh.cells), dtype=np.int8)
    for i, k in enumerate(mesh.cells):
        if k[0] < mesh.max_level and meets(k):
            flags[i] = 1
        elif k[0] > 0 and not meets(parent(k)):
            flags[i] = -1
    return flags
