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
