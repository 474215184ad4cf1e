"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
and its host spacetree logic equals the oracle's (bit-exact integer work)."""
import re
import os

import numpy as np
import pytest

from oracle import mesh as omesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def A():
    from paper_1806_07984_gb300 import ader, build
    build.build()
    ader.lib()
    return ader


def test_missing_library_fails_loudly(A, monkeypatch, tmp_path):
    """Without libader.so every entry point raises: there is no fallback."""
    monkeypatch.setattr(A, "LIB_PATH", str(tmp_path / "libader.so"))
    monkeypatch.setattr(A, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        A.lib()
    with pytest.raises(RuntimeError):
        A.ader_mesh_create(2, (3, 3), 1)


def test_exports_match_header(A):
    header = open(os.path.join(ROOT, "include", "ader.h")).read()
    declared = set(re.findall(r"\b(ader_\w+)\s*\(", header))
    declared -= {"ader_ctx", "ader_mesh"}
    assert declared == set(A.EXPORTS), declared ^ set(A.EXPORTS)
    L = A.lib()
    for name in declared:
        assert hasattr(L, name)
    assert A.ader_error_string(-4) == "non-physical state"


def lib_mesh_state(A, m, dim):
    cells, skel = A.ader_mesh_leaves(m)
    keys = [(int(c[0]), tuple(int(x) for x in c[1:1 + dim])) for c in cells]
    conf, par, kids = A.ader_mesh_faces(m, dim)
    return keys, skel.astype(bool), conf, par, kids


def oracle_face_sets(om):
    conf, parents = om.faces()
    cs = set((om.cells[a], om.cells[b], d) for a, b, d in conf)
    ps = set((om.cells[c], d, s, tuple(om.cells[f] for f, _ in kids)) for c, d, s, kids in parents)
    return cs, ps


def lib_face_sets(keys, conf, par, kids):
    cs = set((keys[a], keys[b], int(d)) for a, b, d in conf)
    ps = set((keys[c], int(d), int(s), tuple(keys[f] for f in kids[i])) for i, (c, d, s) in enumerate(par))
    return cs, ps


def drive(A, dim, base, max_level, centers, radius):
    """Apply the same sphere-flag sequence to both meshes; compare after each."""
    om = omesh.Mesh(dim, (base,) * dim, max_level)
    lm = A.ader_mesh_create(dim, (base,) * dim, max_level)
    try:
        for center in centers:
            keys = lib_mesh_state(A, lm, dim)[0]
            okeys = om.cells
            assert sorted(keys) == okeys
            fl_o = omesh.sphere_flags(om, center, radius)
            fl_l = A.ader_mesh_sphere_flags(lm, center, radius)
            perm = [om.index[k] for k in keys]
            assert np.array_equal(fl_l, fl_o[perm])
            import oracle.basis as ob
            B = ob.Basis(1)
            om.remesh(np.zeros((len(om.cells), 1) + (2,) * dim), fl_o, B)
            A.ader_mesh_adapt(lm, fl_l)
            keys, skel, conf, par, kids = lib_mesh_state(A, lm, dim)
            assert sorted(keys) == om.cells
            oskel = om.skeleton()
            assert np.array_equal(skel, oskel[[om.index[k] for k in keys]])
            assert lib_face_sets(keys, conf, par, kids) == oracle_face_sets(om)
            nconf_sk = sum(1 for a, b, _ in conf if skel[a] and skel[b])
            assert all(skel[a] and skel[b] for a, b, _ in conf[:nconf_sk])
        return len(om.cells)
    finally:
        A.ader_mesh_destroy(lm)


def test_mesh_parity_2d(A):
    centers = [(0.45, 0.55), (0.45, 0.55), (0.6, 0.65), (0.75, 0.8), (0.95, 0.05)]
    assert drive(A, 2, 9, 2, centers, 0.15) > 81


def test_mesh_parity_3d(A):
    centers = [(0.5, 0.5, 0.5), (0.5, 0.5, 0.5), (0.62, 0.6, 0.58), (0.9, 0.1, 0.95)]
    assert drive(A, 3, 3, 2, centers, 0.2) > 27


def test_mesh_parity_deep_2d(A):
    """Three levels with a cascade of balance refinements."""
    centers = [(0.3, 0.3)] * 3 + [(0.32, 0.31), (0.5, 0.5)]
    assert drive(A, 2, 3, 3, centers, 0.02) > 9


def test_mesh_parity_threaded(A):
    """Meshes large enough (> 8,192 leaves) for the multi-threaded host passes
    (depth-first order, face sweep, sphere flags) still equal the oracle's."""
    assert drive(A, 2, 45, 2, [(0.5, 0.5), (0.5, 0.5), (0.58, 0.52)], 0.2) > 16384
    assert drive(A, 3, 20, 1, [(0.5, 0.5, 0.5), (0.6, 0.55, 0.5)], 0.2) > 16384


def test_mesh_single_cell(A):
    lm = A.ader_mesh_create(3, (1, 1, 1), 1)
    try:
        C, nskel, nconf, npar = A.ader_mesh_sizes(lm)
        assert (C, nskel, nconf, npar) == (1, 0, 3, 0)
        conf, _, _ = A.ader_mesh_faces(lm, 3)
        assert conf.tolist() == [[0, 0, 0], [0, 0, 1], [0, 0, 2]]
    finally:
        A.ader_mesh_destroy(lm)


def test_mesh_bad_arguments(A):
    with pytest.raises(A.AderError):
        A.ader_mesh_create(4, (3, 3, 3), 1)
    with pytest.raises(A.AderError):
        A.ader_mesh_create(2, (0, 3, 1), 1)


def test_config_rejected_before_any_device_call(A):
    """ader_init validates the configuration on the host: malformed limiter
    and pipeline settings return ADER_ERR_ARG without a GPU."""
    def cfg(dim, order, limiter):
        c = A.ader_config()
        c.dim, c.order, c.nvar, c.pde = dim, order, dim + 2, A.ADER_EULER
        c.gamma, c.cfl = 1.4, 0.05
        for d in range(3):
            c.base[d], c.lo[d], c.hi[d] = 3, 0.0, 1.0
        c.limiter = limiter
        return c
    bad_chunks = cfg(3, 3, 0)
    bad_chunks.pipeline_chunks = 65
    bad_ctas = cfg(3, 3, 0)
    bad_ctas.pipeline_ctas = -1
    for bad in (cfg(2, 3, 2), cfg(3, 3, -1), bad_chunks, bad_ctas):
        with pytest.raises(A.AderError) as e:
            A.ader_init(bad)
        assert e.value.status == -1


def _pair(A, dim, base, max_level, centers, radius):
    om = omesh.Mesh(dim, (base,) * dim, max_level)
    lm = A.ader_mesh_create(dim, (base,) * dim, max_level)
    import oracle.basis as ob
    for center in centers:
        fl = omesh.sphere_flags(om, center, radius)
        om.remesh(np.zeros((len(om.cells), 1) + (2,) * dim), fl, ob.Basis(1))
        A.ader_mesh_adapt(lm, A.ader_mesh_sphere_flags(lm, center, radius))
    keys = lib_mesh_state(A, lm, dim)[0]
    assert sorted(keys) == om.cells
    return om, lm, keys


@pytest.mark.parametrize("dim,base,centers", [(2, 9, [(0.45, 0.55), (0.45, 0.55)]),
                                              (3, 3, [(0.5, 0.5, 0.5), (0.5, 0.5, 0.5)])])
def test_refine_around_matches_oracle(A, dim, base, centers):
    """The limiter's remesh rule (troubled cells and their face neighbours
    across transitions) equals the oracle's bit for bit."""
    from oracle import limiter as olim
    om, lm, keys = _pair(A, dim, base, 2, centers, 0.15)
    try:
        perm = np.array([om.index[k] for k in keys])
        rng = np.random.default_rng(dim)
        for _ in range(3):
            troubled = rng.random(len(keys)) < 0.05
            got = A.ader_mesh_refine_around(lm, troubled)
            inv = np.argsort(perm)
            want = olim.refine_flags(om, troubled[inv])
            assert np.array_equal(got, want[perm])
    finally:
        A.ader_mesh_destroy(lm)


@pytest.mark.parametrize("K,base,levels", [(1, 3, 2), (3, 3, 2), (8, 3, 2), (8, 20, 1)])
def test_pipeline_lists(A, K, base, levels):
    """Enclave pipeline lists: chunks partition the enclave, every conforming
    face sits after the skeleton faces in the stage of the later chunk of its
    two cells, and every cell is corrected exactly once, in the stage after
    which all its faces are solved.  The base-20 mesh (> 8,192 cells) takes the
    multi-threaded passes of the classification."""
    om, lm, keys = _pair(A, 3, base, levels, [(0.5, 0.5, 0.5)] * levels, 0.2)
    try:
        C = len(keys)
        _, skel = A.ader_mesh_leaves(lm)
        conf_all, par, kids = A.ader_mesh_faces(lm, 3)
        chunk_off, face_off, corr_off, corr_cells, conf, nsk = A.ader_mesh_pipeline(lm, K)
        encl = np.flatnonzero(skel == 0)
        assert chunk_off[0] == 0 and chunk_off[-1] == len(encl) and (np.diff(chunk_off) >= 0).all()
        chunk = -np.ones(C, dtype=int)
        for k in range(K):
            chunk[encl[chunk_off[k]:chunk_off[k + 1]]] = k
        # faces: same set as the mesh's, skeleton faces first, then by stage
        assert sorted(map(tuple, conf.tolist())) == sorted(map(tuple, conf_all.tolist()))
        assert all(skel[a] and skel[b] for a, b, _ in conf[:nsk])
        assert face_off[0] == 0 and face_off[-1] == len(conf) - nsk
        ready = chunk.copy()
        for k in range(K):
            for a, b, _ in conf[nsk + face_off[k]:nsk + face_off[k + 1]]:
                assert max(chunk[a], chunk[b]) == k
                ready[a] = max(ready[a], k)
                ready[b] = max(ready[b], k)
        # cells: a permutation, grouped by ready stage + 1
        assert sorted(corr_cells.tolist()) == list(range(C))
        for g in range(K + 1):
            assert all(ready[c] + 1 == g for c in corr_cells[corr_off[g]:corr_off[g + 1]])
    finally:
        A.ader_mesh_destroy(lm)
