"""The kl-refinement loop (Alg. 2) on the L-shape at its full level L = 7, GPU against the oracle.

Four steps of (FMG solve, estimator, marking of the top 20 %, 2D red-green refinement of the macro
mesh), then a final solve: five solves on macro meshes of 24 to 340 triangles.  At every step the
library's solution and estimates match the oracle's (1e-10, as in the parity tests), the marked
sets are identical, and the two red-green refinements (host C++ in the library, Python in the
oracle) produce the same macro mesh.
"""

import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import workloads as W
from oracle import hhg_oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06049_gb300 as pkg
    pkg.lib()
    return pkg


def test_lshape_l7_kl_loop_matches_oracle(P):
    co, ce, L, f, g, k, _ = W.workload("lshape_l7")
    rg = P.RG2D(co, ce)
    rgo = O.RG2D(co, ce)
    sizes = []
    for step in range(5):
        c, e = rg.mesh()
        co_o, ce_o = rgo.mesh()
        assert np.array_equal(c, co_o) and np.array_equal(e, ce_o)
        sizes.append(len(e))
        mesh = P.Mesh(c, e, L)
        x = mesh.level_coords(L)
        mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
        u = mesh.solve()
        est = mesh.estimate(1)
        h = O.Hierarchy(co_o, ce_o, L)
        uo, ws, _ = O.fmg(O.Problem(h, f, g), 2, 2, 1)
        eo = O.estimate(h, uo, ws, 1)
        dist, idx = cKDTree(h.levels[L].x).query(x)
        assert dist.max() < 1e-9
        scale = np.abs(uo).max()
        assert np.abs(u - uo[idx]).max() <= TOL * scale
        u_T = np.sqrt(O.local_mass_sq(h.levels[L], uo, h.n_cells))
        assert np.all(np.abs(est["eta_T"] - eo["eta_T"]) <= TOL * u_T)
        u_glob = math.sqrt(float((u_T ** 2).sum()))
        assert abs(est["eta_j"] - eo["eta_j"]) <= 10 * TOL * u_glob
        mesh.close()
        if step == 4:
            break
        mk = P.mark(est["eta_T"], 0.2)
        assert np.array_equal(mk, O.mark_top_fraction(eo["eta_T"], 0.2))
        rg.refine(mk)
        rgo.refine(mk)
    assert sizes[0] == 24 and all(b > a for a, b in zip(sizes, sizes[1:])), sizes


def test_cube_kl_loop_3d_matches_oracle(P):
    """The 3D kl step (Alg. 2 with Alg. 3): on 48 Kuhn tets at L = 3, three steps of (FMG solve,
    estimator, marking of the top 12.5 %, 3D red-green refinement) and a final solve, GPU against
    the oracle: solutions and estimates to 1e-10, identical markings, identical macro meshes (the
    refined meshes have tets of every orientation and general shape: full 15-point stencils)."""
    co, ce = W.cube_mesh(2)
    L = 3
    f = lambda x: np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]) + x[:, 2]
    g = lambda x: 0.1 * x[:, 0] - x[:, 2] * x[:, 1]
    rg = P.RG3D(co, ce)
    rgo = O.RG3D(co, ce)
    sizes = []
    for step in range(4):
        c, e = rg.mesh()
        co_o, ce_o = rgo.mesh()
        assert np.array_equal(c, co_o) and np.array_equal(e, ce_o)
        sizes.append(len(e))
        mesh = P.Mesh(c, e, L)
        x = mesh.level_coords(L)
        mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
        u = mesh.solve()
        est = mesh.estimate(1)
        h = O.Hierarchy(co_o, ce_o, L)
        uo, ws, _ = O.fmg(O.Problem(h, f, g), 2, 2, 1)
        eo = O.estimate(h, uo, ws, 1)
        dist, idx = cKDTree(h.levels[L].x).query(x)
        assert dist.max() < 1e-9
        assert np.abs(u - uo[idx]).max() <= TOL * np.abs(uo).max()
        u_T = np.sqrt(O.local_mass_sq(h.levels[L], uo, h.n_cells))
        assert np.all(np.abs(est["eta_T"] - eo["eta_T"]) <= TOL * u_T)
        mesh.close()
        if step == 3:
            break
        mk = rg.mark_refine(est["eta_T"], 0.125)
        assert np.array_equal(mk, O.mark_top_fraction(eo["eta_T"], 0.125))
        rgo.refine(mk)
    assert sizes[0] == 48 and all(b > a for a, b in zip(sizes, sizes[1:])), sizes
