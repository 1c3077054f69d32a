"""3D red-green refinement (Alg. 3, Sec. 3): the oracle pinned by mesh invariants, the library's
host implementation bit-exact against it (no GPU needed)."""

from collections import Counter

import numpy as np
import pytest

import workloads as W
from oracle import hhg_oracle as O

FACES = ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def signed_volumes(co, ce):
    X = co[ce]
    return np.einsum("ij,ij->i", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0]) / 6


def quality(co, ce):
    X = co[ce]
    hmax = np.max([np.linalg.norm(X[:, a] - X[:, b], axis=1) for a, b in EDGES], axis=0)
    return np.abs(signed_volumes(co, ce)) / hmax ** 3


def check_conforming(co, ce, on_boundary):
    faces = Counter()
    for t in ce:
        for f in FACES:
            faces[tuple(sorted(t[list(f)]))] += 1
    assert max(faces.values()) <= 2
    for f, k in faces.items():
        if k == 1:
            assert on_boundary(co[list(f)]), f
    assert len(np.unique(ce)) == len(co)  # every vertex is used


def cube_boundary(P):
    return any(np.all(np.abs(P[:, d]) < 1e-12) or np.all(np.abs(P[:, d] - 1) < 1e-12) for d in range(3))


def fichera_boundary(P):
    """The unit cube without the octant [0, 1/2]^3: its outer faces and the three re-entrant ones."""
    if cube_boundary(P):
        return True
    for d in range(3):
        others = [q for q in range(3) if q != d]
        if np.all(np.abs(P[:, d] - 0.5) < 1e-12) and np.all(P[:, others] <= 0.5 + 1e-12):
            return True
    return False


MESHES = {"cube": (lambda: W.cube_mesh(2), cube_boundary), "fichera": (W.fichera_mesh, fichera_boundary)}


@pytest.mark.parametrize("name", list(MESHES))
def test_rg3d_oracle_invariants(name):
    """Conforming (every face shared by two tets or on the domain boundary), volume conserved with
    each child keeping its parent's orientation, marked tets red-refined, shape quality bounded
    across steps (greens reverted), and a step without marks reproduces the mesh."""
    mk, on_bnd = MESHES[name]
    co, ce = mk()
    rg = O.RG3D(co, ce)
    v0 = signed_volumes(co, ce)
    q0 = quality(co, ce).min()
    rng = np.random.default_rng(5)
    for step in range(3):
        c, e = rg.mesh()
        marked = rng.random(len(e)) < 0.1
        marked[0] = True
        # (a marked green child marks its green parent instead: only regular tets are checked)
        regular = marked & np.array([t[1] is None for t in rg.tets])
        parents = c[e[regular]]
        vol_marked = np.abs(signed_volumes(c, e))[regular]
        rg.refine(marked)
        c2, e2 = rg.mesh()
        check_conforming(c2, e2, on_bnd)
        vol = signed_volumes(c2, e2)
        assert abs(np.abs(vol).sum() - np.abs(v0).sum()) < 1e-12
        assert abs(vol.sum() - v0.sum()) < 1e-12  # orientations kept (the inputs mix both signs)
        assert np.all(np.abs(vol) > 0)
        assert quality(c2, e2).min() >= 0.25 * q0 - 1e-12
        # a marked tet was red-refined: the tets inside it (their centroids strictly inside) fill
        # its volume and none is larger than an eighth of it
        cent = c2[e2].mean(axis=1)
        for X, vm in zip(parents, vol_marked):
            J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
            lam = np.linalg.solve(J, (cent - X[0]).T).T
            inside = np.all(lam > 1e-12, axis=1) & (lam.sum(axis=1) < 1 - 1e-12)
            assert abs(np.abs(vol[inside]).sum() - vm) < 1e-12 * max(1.0, vm)
            assert np.abs(vol[inside]).max() <= vm / 8 + 1e-15
    before = rg.mesh()
    rg.refine(np.zeros(len(rg.tets), dtype=bool))
    after = rg.mesh()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


def test_rg3d_green_types():
    """One split edge -> 2 children, two opposite edges -> 4, the three edges of one face -> 4; a
    single marked tet of a 2-tet mesh leaves its neighbour with one fully split face."""
    co = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=float)
    ce = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    rg = O.RG3D(co, ce)
    rg.refine([True, False])
    fam = Counter(id(t[1]) if t[1] is not None else None for t in rg.tets)
    sizes = sorted(n for k, n in fam.items() if k is not None)
    assert sizes == [4]  # the neighbour: three edges of the shared face split -> 4 green children
    c, e = rg.mesh()
    assert len(e) == 8 + 4
    check_conforming(c, e, lambda P: True)


def test_rg3d_library_matches_oracle_bit_exactly():
    """The library's host implementation (hhg_rg3d_*) against the oracle: identical vertex
    coordinates, cell lists and markings over three steps on two meshes."""
    import paper_2508_06049_gb300 as P
    try:
        P.lib()
    except ImportError:
        pytest.skip("libhhg.so not built")
    for mk in (lambda: W.cube_mesh(2), W.fichera_mesh):
        co, ce = mk()
        a, b = P.RG3D(co, ce), O.RG3D(co, ce)
        rng = np.random.default_rng(7)
        for step in range(3):
            eta = rng.random(len(b.tets))
            ma = a.mark_refine(eta, 0.125)
            mb = O.mark_top_fraction(eta, 0.125)
            b.refine(mb)
            assert np.array_equal(ma, mb)
            ca, ea = a.mesh()
            cb, eb = b.mesh()
            assert np.array_equal(ca, cb) and np.array_equal(ea, eb)


def test_rg_libraries_reject_bad_meshes():
    """hhg_rg2d_create / hhg_rg3d_create: vertex ids out of range -> HHG_ERR_ARG (1); a cell with a
    repeated vertex or zero measure -> HHG_ERR_MESH (2); a refine step with a NULL mark array or a
    size query without arrays behaves as declared."""
    import paper_2508_06049_gb300 as P
    try:
        P.lib()
    except ImportError:
        pytest.skip("libhhg.so not built")
    co3, ce3 = W.cube_mesh(1)
    bad = ce3.copy()
    bad[0, 3] = len(co3)
    with pytest.raises(P.HHGError) as e:
        P.RG3D(co3, bad)
    assert e.value.status == 1
    rep = ce3.copy()
    rep[1, 2] = rep[1, 0]
    with pytest.raises(P.HHGError) as e:
        P.RG3D(co3, rep)
    assert e.value.status == 2
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=float)
    with pytest.raises(P.HHGError) as e:
        P.RG3D(flat, np.array([[0, 1, 2, 3]]))
    assert e.value.status == 2
    co2, ce2 = W.square_mesh(2)
    rep2 = ce2.copy()
    rep2[0, 1] = rep2[0, 2]
    with pytest.raises(P.HHGError) as e:
        P.RG2D(co2, rep2)
    assert e.value.status == 2
    line = np.array([[0, 0], [1, 0], [2, 0]], dtype=float)
    with pytest.raises(P.HHGError) as e:
        P.RG2D(line, np.array([[0, 1, 2]]))
    assert e.value.status == 2
    rg = P.RG3D(co3, ce3)
    assert P.lib().hhg_rg3d_refine(rg._h, None) == 1
    c, e3 = rg.mesh()
    assert np.array_equal(c, co3) and np.array_equal(e3, ce3)
