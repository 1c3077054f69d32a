"""Host pieces of the estimator study (`bench.py --program effectivity`): the quadrature rule, the
micro-triangle enumeration of the packed closure layout, the local L2 error norms and the
idealised constants of Theorem 4.1 (no GPU needed)."""

import math
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

torch = pytest.importorskip("torch")


def test_radon_rule_is_exact_to_degree_five():
    # reference triangle (0,0), (1,0), (0,1): int x^a y^b = a! b! / (a + b + 2)!
    pts, w = bench.radon7()
    assert abs(sum(w) - 1) < 1e-15
    for a in range(6):
        for b in range(6 - a):
            q = sum(wi * (p[1] ** a) * (p[2] ** b) for p, wi in zip(pts, w)) * 0.5
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(q - exact) < 1e-15, (a, b)
    # not exact at degree 6 (so the test above is not vacuous)
    q6 = sum(wi * p[1] ** 6 for p, wi in zip(pts, w)) * 0.5
    assert abs(q6 - math.factorial(6) / math.factorial(8)) > 1e-6


@pytest.mark.parametrize("n", [1, 2, 4, 16])
def test_micro_triangles_tile_the_macro_triangle(n):
    tri = bench.micro_triangles(n)
    assert tri.shape == (n * n, 3)
    P = np.array([(i, j) for j in range(n + 1) for i in range(n + 1 - j)], dtype=float)
    assert tri.min() == 0 and tri.max() == len(P) - 1
    X = P[tri]
    d1, d2 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    assert np.all(det == 1)                        # counter-clockwise, area 1/2 each
    edges = {}
    for t in tri:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            e = tuple(sorted((t[a], t[b])))
            edges[e] = edges.get(e, 0) + 1
    boundary = sum(1 for k in edges.values() if k == 1)
    assert max(edges.values()) <= 2 and boundary == 3 * n   # conforming, the macro edges once


def _closure_coords(co, ce, n):
    xs = []
    for cv in ce:
        x0 = co[cv[0]]
        J = np.stack([co[cv[1]] - x0, co[cv[2]] - x0], 1)
        for j in range(n + 1):
            for i in range(n + 1 - j):
                xs.append(x0 + J @ np.array([i, j]) / n)
    return np.array(xs)


def test_local_l2_errors_closed_forms():
    co = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    ce = np.array([[0, 1, 2], [0, 2, 3]])
    n = 4
    x = torch.from_numpy(_closure_coords(co, ce, n))
    tri = bench.micro_triangles(n)
    Nt = (n + 1) * (n + 2) // 2
    # a linear function is reproduced exactly by its interpolant
    lin = lambda y: 0.3 + 2.0 * y[:, 0] - 1.5 * y[:, 1]
    e2 = bench.local_l2_errors_sq(x, lin(x), lin, tri, Nt, 2)
    assert float(e2.abs().max()) < 1e-28
    # u_h = 0 against u = x^2: int over the lower triangle (y <= x) of x^4 = 1/6, over the upper 1/30
    sq = lambda y: y[:, 0] ** 2
    e2 = bench.local_l2_errors_sq(x, torch.zeros(len(x), dtype=torch.float64), sq, tri, Nt, 2)
    assert abs(float(e2[0]) - 1 / 6) < 1e-14 and abs(float(e2[1]) - 1 / 30) < 1e-14
    # u_h = I(x^2) against u = x^2
    e2 = bench.local_l2_errors_sq(x, sq(x), sq, tri, Nt, 2, chunk_cells=1)
    h = 1.0 / n
    # every micro triangle lies in a strip a <= x <= a + h with its vertices on the strip's edges, so
    # there x^2 - I x^2 = (x - a)(x - a - h); over the unit square: n strips of h^5 / 30 each
    total = float(e2.sum())
    assert abs(total - h ** 4 / 30) < 1e-15


def test_theorem_bounds_reproduce_the_printed_constants():
    # Tables 1-2: theta = 2^-2 (waves) and 2^-(4/3) (L-shape), j = 1..4, two decimals
    waves = [(0.53, 1.67), (0.80, 1.24), (0.93, 1.08), (0.98, 1.02)]
    lshape = [(0.31, 2.32), (0.53, 1.76), (0.72, 1.37), (0.85, 1.18)]
    for theta, table in ((2.0 ** -2, waves), (2.0 ** (-4 / 3), lshape)):
        for j, (c1, c2) in enumerate(table, start=1):
            a, b = bench.theorem_bounds(theta, j)
            assert round(a, 2) == c1 and round(b, 2) == c2


class _OracleMesh:
    """Test double of the library's Mesh for the study programs' host logic: the same per-cell
    closure layout (coordinates, solution, stored w_0), computed with the oracle."""

    def __init__(self, c, e, L, stream=None):
        from oracle import hhg_oracle as O
        self.O = O
        self.c, self.e, self.L = np.asarray(c, dtype=float), np.asarray(e), L
        self.h = O.Hierarchy(self.c, self.e, L)
        n = 1 << L
        self.Nt = (n + 1) * (n + 2) // 2
        self.info = type("Info", (), {"n_unknowns": int(self.h.levels[L].free.sum())})()

    def n_nodes(self, level):
        assert level == self.L
        return self.Nt * len(self.e)

    def level_coords(self, level, out):
        n = 1 << level
        ij = np.array([(i, j) for j in range(n + 1) for i in range(n + 1 - j)], dtype=float) / n
        X0 = self.c[self.e[:, 0]]
        J = np.stack([self.c[self.e[:, 1]] - X0, self.c[self.e[:, 2]] - X0], axis=2)
        X = X0[:, None, :] + np.einsum("cra,pa->cpr", J, ij)
        self.X = X.reshape(-1, 2)
        out.copy_(torch.from_numpy(self.X))

    def _to_closure(self, vals, level):
        from scipy.spatial import cKDTree
        d, idx = cKDTree(self.h.levels[level].x).query(self.X)
        assert d.max() < 1e-12
        return torch.from_numpy(vals[idx])

    def set_data(self, f, g):
        from scipy.spatial import cKDTree
        tree = cKDTree(self.X)
        fv, gv = f.numpy().copy(), g.numpy().copy()

        def lookup(vals):
            return lambda Y: vals[tree.query(Y)[1]]
        self.prob = self.O.Problem(self.h, lookup(fv), lookup(gv))

    def solve(self, prm, out):
        self.uo, self.ws, _ = self.O.fmg(self.prob, prm.nu, prm.pre, prm.post, prm.n_extra)
        out.copy_(self._to_closure(self.uo, self.L))

    def estimate(self, j, want_local=True):
        return self.O.estimate(self.h, self.uo, self.ws, j)

    def get_vector(self, which, level, out):
        assert which == 1 and level == self.L - 1
        out.copy_(self._to_closure(self.ws[level], self.L))

    def close(self):
        pass


def _stand_in():
    import types
    from oracle import hhg_oracle as O
    return types.SimpleNamespace(solve_params=lambda **kw: types.SimpleNamespace(**kw), RG2D=O.RG2D,
                                 Mesh=_OracleMesh, mark=O.mark_top_fraction)


def test_effectivity_study_runs_end_to_end():
    """Host logic of `--program effectivity` on a stand-in library: rows for every step, effectivity
    = eta_j / ||e||, worst case = largest |log|, the paper's values and C_1, C_2 attached."""
    res = bench.effectivity_study(_stand_in(), "cpu", L=5, K=1, nus=(2,), n_extra=2)
    assert set(res) == {"waves2d_nu2", "lshape_nu2"}
    for key, v in res.items():
        assert [r["k"] for r in v["rows"]] == [0, 1]
        assert v["rows"][1]["cells"] > v["rows"][0]["cells"]
        for r in v["rows"]:
            assert np.allclose(r["effectivity"], np.array(r["eta"]) / r["l2_error"])
        for jj in range(4):
            vals = [r["effectivity"][jj] for r in v["rows"]]
            assert abs(math.log(v["worst_effectivity"][jj])) == max(abs(math.log(g)) for g in vals)
        assert len(v["paper_worst_effectivity"]) == 4 and len(v["C1_C2"]) == 4


def test_kl_compare_study_runs_end_to_end():
    """Host logic of `--program kl_compare` on a stand-in library at L = 3, K = 2: the three schemes
    report their final grids, Alg. 2 its history, and rho = (cells 4^L / cells_0) ||e_h|| / ||e_H||."""
    res = bench.kl_compare_study(_stand_in(), "cpu", L=3, K=2, n_extra=2)
    for name, r in res.items():
        assert r["uniform"]["cells"] == r["coarse_cells"]
        assert r["alg1"]["cells"] > r["coarse_cells"] and r["alg2"]["cells"] > r["coarse_cells"]
        assert len(r["alg2"]["history"]) == 3
        for key in ("uniform", "alg1", "alg2"):
            s = r[key]
            assert s["rho"] == pytest.approx(s["cells"] * 4 ** 3 / r["coarse_cells"] * s["l2_error"] / r["coarse_error"])
