"""Shared helpers for the oracle tests: meshes and seeded states in the
oracle's layout u[c, var, *nodes]."""
import numpy as np

from oracle import basis, mesh as meshmod
import workloads


def state_from(mesh, B, fn):
    coords = mesh.node_coords(B.xi)
    q = fn(coords)                                # (m, C, *nodes)
    return np.ascontiguousarray(np.moveaxis(q, 0, 1))


def refined_mesh(dim, base, max_level, center, radius, rounds=None):
    """Base grid refined around a ball by repeated sphere flags."""
    m = meshmod.Mesh(dim, (base,) * dim, max_level)
    B0 = basis.Basis(1)
    u = np.zeros((len(m.cells), 1) + (2,) * dim)
    for _ in range(max_level if rounds is None else rounds):
        flags = meshmod.sphere_flags(m, center, radius)
        u = m.remesh(u, flags, B0)
    return m


def random_state(mesh, B, pde_name, seed):
    rng = np.random.default_rng(seed)
    shape = (len(mesh.cells),) + (B.n,) * mesh.dim
    if pde_name == "euler":
        q = workloads.random_euler(rng, mesh.dim, shape)
    else:
        q = workloads.random_acoustics(rng, mesh.dim, shape)
    return np.ascontiguousarray(np.moveaxis(q, 0, 1))
