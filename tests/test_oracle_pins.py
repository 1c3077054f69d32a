"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

None of these tests compares the oracle with itself: every expected value is a closed form,
an invariant, a textbook/library routine on a tiny case, or a number printed in the paper.
"""

import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import hhg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hier(name, L, **kw):
    co, ce, _, f, g, k, ue = W.workload(name, L)
    h = O.Hierarchy(co, ce, L, k=k, **kw)
    return h, f, g, ue


# ---------------------------------------------------------------- refinement (Sec. 2)

@pytest.mark.parametrize("m,L", [(2, 4), (3, 2)])
def test_square_node_and_element_counts(m, L):
    co, ce = W.square_mesh(m)
    h = O.Hierarchy(co, ce, L)
    for l, lev in enumerate(h.levels):
        assert len(lev.keys) == (m * 2 ** l + 1) ** 2
        assert len(lev.elems) == len(ce) * 4 ** l


def test_cube_node_and_element_counts():
    co, ce = W.cube_mesh(2)
    h = O.Hierarchy(co, ce, 2)
    for l, lev in enumerate(h.levels):
        assert len(lev.keys) == (2 * 2 ** l + 1) ** 3
        assert len(lev.elems) == len(ce) * 8 ** l


def test_node_coordinates_form_uniform_grid():
    co, ce = W.cube_mesh(2)
    h = O.Hierarchy(co, ce, 2)
    x = h.levels[2].x * 8
    assert np.allclose(x, np.round(x), atol=1e-12)
    assert len({tuple(p) for p in np.round(x).astype(int)}) == 9 ** 3


def test_bey_refinement_is_the_kuhn_lattice():
    """Bey's rule on the reference tet gives the Freudenthal subdivision of the Kuhn simplex
    0 <= y1 <= y2 <= y3 <= n in y = (i, i+j, i+j+k) (a structural fact the lattice layout uses)."""
    co = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    h = O.Hierarchy(co, np.array([[0, 1, 2, 3]]), 3)
    n = 8
    lev = h.levels[3]
    p = np.round(lev.x * n).astype(int)  # lattice coords (i, j, k) for this unit macro
    got = {frozenset(tuple(p[v]) for v in e) for e in lev.elems}
    want = set()
    for c in itertools.product(range(n), repeat=3):
        for s in itertools.permutations(range(3)):
            y = [list(c)]
            cur = list(c)
            for a in s:
                cur = cur[:]
                cur[a] += 1
                y.append(cur)
            if all(0 <= v[0] <= v[1] <= v[2] <= n for v in y):
                want.add(frozenset((v[0], v[1] - v[0], v[2] - v[1]) for v in y))
    assert got == want


# ---------------------------------------------------------------- assembly (Eq. 5.1)

@pytest.mark.parametrize("name,L,area", [("square_l4", 3, 1.0), ("lshape_l7", 3, 3.0),
                                         ("cube384_l6", 2, 1.0), ("fichera336_l6", 1, 7.0 / 8.0)])
def test_mass_matrix_total_is_domain_measure(name, L, area):
    h, *_ = _hier(name, L)
    for lev in h.levels:
        assert abs(lev.M.sum() - area) < 1e-13 * max(1, area)


@pytest.mark.parametrize("name,L", [("square_l4", 3), ("cube384_l6", 2), ("cube3072_l7", 1)])
def test_stiffness_symmetric_with_zero_row_sums(name, L):
    h, *_ = _hier(name, L)
    for lev in h.levels:
        A = lev.A
        assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
        assert np.abs(A @ np.ones(A.shape[0])).max() <= 1e-13 * abs(A).max()
        # positive diagonal, non-positive couplings for these (non-obtuse) meshes
        assert (A.diagonal() > 0).all()


@pytest.mark.parametrize("dim", [2, 3])
def test_kuhn_split_gives_finite_difference_laplacian(dim):
    """Right-isosceles triangles / Kuhn tets: P1 stiffness = (2d, -1 on axis neighbours) h^(d-2)."""
    co, ce = (W.square_mesh(2) if dim == 2 else W.cube_mesh(2))
    L = 2
    h = O.Hierarchy(co, ce, L)
    lev = h.levels[L]
    hh = 1.0 / (2 * 2 ** L)
    s = hh ** (dim - 2)
    grid = np.round(lev.x / hh).astype(int)
    index = {tuple(p): i for i, p in enumerate(grid)}
    A = lev.A.tocsr()
    for i, p in enumerate(grid):
        if np.any(p == 0) or np.any(p == 2 * 2 ** L):
            continue
        want = {i: 2 * dim * s}
        for a in range(dim):
            for sg in (-1, 1):
                q = list(p)
                q[a] += sg
                want[index[tuple(q)]] = -s
        row = A.getrow(i)
        got = {j: v for j, v in zip(row.indices, row.data) if abs(v) > 1e-13}
        assert got.keys() == want.keys()
        for j in want:
            assert abs(got[j] - want[j]) < 1e-12 * s


@pytest.mark.parametrize("name,L", [("lshape_l7", 3), ("cube3072_l7", 2), ("fichera336_l6", 2)])
def test_galerkin_identity(name, L):
    """Nested P1 spaces: P^T A_l P = A_{l-1} and P^T M_l P = M_{l-1} (coefficient constant per macro)."""
    h, *_ = _hier(name, L)
    for l in range(1, L + 1):
        P = h.levels[l].P
        for op in ("A", "M"):
            fine = getattr(h.levels[l], op)
            coarse = getattr(h.levels[l - 1], op)
            diff = abs(P.T @ fine @ P - coarse).max()
            assert diff <= 1e-13 * abs(coarse).max(), (op, l, diff)


@pytest.mark.parametrize("name,L", [("square_l4", 3), ("cube384_l6", 2)])
def test_restricted_rhs_is_the_load_vector_of_the_fine_interpolant(name, L):
    """The restricted right-hand sides b_l = I^T b_{l+1}, b_L = M_L f_L: (i) for f the interpolant of
    a level-m function (f_L = I ... I f_m) they equal the injected b_l = M_l f_l on every level l >= m
    (Galerkin identity I^T M_{l+1} I = M_l; there f_l is the interpolant too), and a generic f makes
    them differ below level L; (ii) on every level,
    b_l^T v_l = b_L^T (I ... I v_l) for any level-l vector v_l (b_l tests the level-L load vector with
    the level-l hat functions written in the level-L basis)."""
    h, *_ = _hier(name, L)
    rng = np.random.default_rng(4)
    m = 1
    fm = rng.standard_normal(len(h.levels[m].keys))
    fL = fm
    for l in range(m + 1, L + 1):
        fL = h.levels[l].P @ fL
    zero = lambda x: np.zeros(len(x))
    pr = O.Problem(h, fL, zero, rhs="restricted")
    pi = O.Problem(h, fL, zero, rhs="injected")
    for l in range(L + 1):
        scale = np.abs(pi.b[l]).max()
        diff = np.abs(pr.b[l] - pi.b[l]).max()
        if l >= m:
            assert diff <= 1e-13 * scale, (l, diff)
    # a generic f: the restricted and injected coarse right-hand sides differ below level L
    x = h.levels[L].x
    pr2 = O.Problem(h, lambda y: np.exp(3 * y[:, 0]) * np.cos(5 * y[:, 1]), zero, rhs="restricted")
    pi2 = O.Problem(h, lambda y: np.exp(3 * y[:, 0]) * np.cos(5 * y[:, 1]), zero, rhs="injected")
    assert np.array_equal(pr2.b[L], pi2.b[L])
    assert np.abs(pr2.b[L - 1] - pi2.b[L - 1]).max() > 1e-6 * np.abs(pi2.b[L - 1]).max()
    for l in range(L + 1):
        v = rng.standard_normal(len(h.levels[l].keys))
        vL = v
        for q in range(l + 1, L + 1):
            vL = h.levels[q].P @ vL
        lhs, rhs = float(pr2.b[l] @ v), float(pr2.b[L] @ vL)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs)), (l, lhs, rhs)
    with pytest.raises(ValueError):
        O.Problem(h, zero, zero, rhs="other")


def test_interpolation_reproduces_linear_functions():
    h, *_ = _hier("cube3072_l7", 2)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(4)
    for l in range(1, 3):
        xc, xf = h.levels[l - 1].x, h.levels[l].x
        vc = c[0] + xc @ c[1:]
        vf = c[0] + xf @ c[1:]
        assert np.abs(h.levels[l].P @ vc - vf).max() < 1e-13


# ---------------------------------------------------------------- solver (Alg. 4)

def test_linear_solution_is_reproduced_and_estimate_vanishes():
    co, ce = W.lshape_mesh()
    L = 4
    h = O.Hierarchy(co, ce, L)
    g = lambda x: 0.3 - 1.7 * x[:, 0] + 0.9 * x[:, 1]
    prob = O.Problem(h, lambda x: np.zeros(len(x)), g)
    u, ws, _ = O.fmg(prob, 2, 2, 1)
    assert np.abs(u - g(h.levels[L].x)).max() < 1e-12
    est = O.estimate(h, u, ws, 1)
    assert est["err_l"] < 1e-12 and est["eta_T"].max() < 1e-12


@pytest.mark.parametrize("name,L,extra", [("square_l4", 3, 30), ("cube384_l6", 2, 40),
                                          ("cube3072_l7", 2, 120)])
def test_fmg_plus_vcycles_converges_to_direct_solve(name, L, extra):
    # k log-uniform over four decades (cube3072) contracts at ~0.75 per V-cycle: more cycles
    h, f, g, _ = _hier(name, L)
    prob = O.Problem(h, f, g)
    u, _, _ = O.fmg(prob, 2, 2, 1, n_extra=extra)
    ex = O.exact_solve(prob)
    assert np.abs(u - ex).max() <= 1e-12 * max(1.0, np.abs(ex).max())


def test_coarse_level_fmg_is_exact():
    """On level 0 the FMG V-cycle is the direct solve: compare with a dense library solve."""
    h, f, g, _ = _hier("fichera336_l6", 1)
    prob = O.Problem(h, f, g)
    _, _, us = O.fmg(prob, 1, 2, 1)
    lev = h.levels[0]
    F = lev.free
    A = lev.A.toarray()
    want = np.zeros(len(F))
    want[F] = np.linalg.solve(A[np.ix_(F, F)], prob.b[0][F])
    assert np.abs(us[0] - want).max() < 1e-13 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("name,L,bound", [("square_l4", 5, 0.2), ("lshape_l7", 5, 0.2), ("cube384_l6", 3, 0.4)])
def test_vcycle_contraction(name, L, bound):
    """A working V(2,1) cycle contracts the residual by a mesh-independent factor well below 1
    (measured ~0.1 in 2D; ~0.3 in 3D where P1 interpolation on Kuhn tets is less accurate)."""
    h, f, g, _ = _hier(name, L)
    prob = O.Problem(h, f, g)
    lev = h.levels[L]
    rng = np.random.default_rng(0)
    u = np.where(lev.dirichlet, prob.g[L], rng.standard_normal(len(lev.keys)))
    norms = []
    for _ in range(5):
        norms.append(np.linalg.norm(O.residual(lev, u, prob.b[L])))
        O.vcycle(prob, L, u, prob.b[L], 2, 1)
    rates = [norms[i + 1] / norms[i] for i in range(1, 4)]
    assert max(rates) < bound, rates


def test_smoother_stage_equals_true_gauss_seidel_when_colours_are_valid():
    """Right-isosceles triangles: every macro-interior colour stage has no internal couplings, so
    the Jacobi-within-stage update is exactly sequential Gauss-Seidel over that stage.  (Odd
    edge nodes next to a shared macro vertex do couple across edges: that stage is Jacobi.)"""
    h, f, g, _ = _hier("square_l4", 4)
    lev = h.levels[4]
    cell_stages = range(3, len(lev.stages))
    for s in cell_stages:
        idx = lev.stages[s]
        sub = lev.A[idx][:, idx].tocoo()
        off = np.abs(sub.data[sub.row != sub.col])
        assert off.size == 0 or off.max() < 1e-13, s
    prob = O.Problem(h, f, g)
    rng = np.random.default_rng(1)
    A = lev.A.tocsr()
    for s in cell_stages:
        idx = lev.stages[s]
        u = np.where(lev.dirichlet, 0.0, rng.standard_normal(len(lev.keys)))
        u1 = u.copy()
        u1[idx] += (prob.b[4][idx] - lev.stage_rows[s] @ u1) / lev.stage_diag[s]
        u2 = u.copy()
        for i in idx:
            u2[i] += (prob.b[4][i] - A.getrow(i) @ u2)[0] / A[i, i]
        assert np.abs(u1 - u2).max() < 1e-13


def test_face_block_is_per_face_gauss_seidel_with_frozen_surroundings():
    """3D face block, written out node by node: for every macro face, sequential Gauss-Seidel over
    its nodes in colour order, reading its own nodes at their current values and every other node
    at its value from the start of the block.  Face and colour are recomputed here from the node
    keys (vertex ids and barycentric weights), not taken from the oracle's stage data."""
    co, ce = W.cube_mesh(2)
    h = O.Hierarchy(co, ce, 3, k=W.coeff_uniform(len(ce), seed=5))
    lev = h.levels[3]
    A = lev.A.tocsr()
    keys = lev.keys
    g, w = keys[:, 0::2], keys[:, 1::2]
    nv = (w > 0).sum(axis=1)
    face = {}
    for i in np.nonzero((nv == 3) & lev.free)[0]:
        fk = tuple(sorted(g[i, :3]))
        col = (w[i, 1] + 2 * w[i, 2]) % 3
        face.setdefault(fk, []).append((col, i))
    assert len(face) > 4
    rng = np.random.default_rng(2)
    u = np.where(lev.dirichlet, 0.0, rng.standard_normal(len(keys)))
    rhs = rng.standard_normal(len(keys))
    # stages before the face block (vertices, edges), then the block literally
    ref = u.copy()
    for s in range(3):
        idx = lev.stages[s]
        ref[idx] += (rhs[idx] - A[idx] @ ref) / A.diagonal()[idx]
    frozen = ref.copy()
    for fk, nodes in face.items():
        mine = np.zeros(len(keys), dtype=bool)
        mine[[i for _, i in nodes]] = True
        for col in range(3):
            for c, i in nodes:
                if c != col:
                    continue
                row = A.getrow(i)
                vals = np.where(mine[row.indices], ref[row.indices], frozen[row.indices])
                ref[i] += (rhs[i] - row.data @ vals) / A[i, i]
    # the oracle's sweep, stopped after the face block
    got = u.copy()
    stages, lev.stages = lev.stages, lev.stages[:6]
    try:
        O.smooth(lev, got, rhs)
    finally:
        lev.stages = stages
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------- discretisation (Sec. 5)

def _inv_inf(lev):
    A = lev.A.toarray()[np.ix_(lev.free, lev.free)]
    return float(np.abs(np.linalg.inv(A)).sum(axis=1).max())


@pytest.mark.parametrize("mesh,L,lo,hi", [
    ("square", 3, 1.0, 1.5), ("lshape", 2, 1.0, 1.5), ("cube", 2, 1.0, 1.5),
    ("cube_k4", 2, 1.0, 16.0),
])
def test_inverse_norm_grows_like_the_level_volume(mesh, L, lo, hi):
    """The range bound of binary16 correction storage: |A_l^{-1}|_inf / (2^{l d} |A_0^{-1}|_inf)
    stays within [lo, hi] (the discrete Green's function of a nested P1 level grows like 2^{l d}).
    Dense inverses of the assembled free-node operators on the first levels.  With a constant
    coefficient the ratio stays near 1 (at most 1.18 / 1.21 / 1.32 on these meshes); with k_T
    log-uniform over four decades level 0 does not resolve the coefficient jumps and the ratio
    levels off near 15 on this 384-tet cube (5.3, 13.2, 14.1, 14.5 on levels 1-4)."""
    if mesh == "square":
        co, ce = W.square_mesh(2)
        k = None
    elif mesh == "lshape":
        co, ce = W.lshape_mesh()
        k = None
    elif mesh == "cube":
        co, ce = W.cube_mesh(2)
        k = None
    else:
        co, ce = W.cube_mesh(4)
        k = W.coeff_loguniform(len(ce), seed=0)
    h = O.Hierarchy(co, ce, L, k=k)
    d = h.dim
    a0 = _inv_inf(h.levels[0])
    for l in range(1, L + 1):
        r = _inv_inf(h.levels[l]) / (2.0 ** (l * d) * a0)
        assert lo <= r <= hi, (l, r)


def _errors(name, Ls, fn=None):
    out = []
    for L in Ls:
        h, f, g, ue = _hier(name, L)
        prob = O.Problem(h, f, g)
        u, _, _ = O.fmg(prob, 2, 2, 1, n_extra=6)
        out.append(math.sqrt(O.l2_error_sq(h, u, ue)))
    return np.array(out)


def test_manufactured_2d_second_order():
    e = _errors("square_l4", [3, 4, 5, 6])
    r = e[:-1] / e[1:]
    assert np.all(np.abs(r[1:] - 4.0) < 0.25), r


def test_manufactured_3d_second_order():
    e = []
    for L in (2, 3, 4):
        co, ce = W.cube_mesh(1)
        h = O.Hierarchy(co, ce, L)
        prob = O.Problem(h, W.sin_product_f, lambda x: np.zeros(len(x)))
        u, _, _ = O.fmg(prob, 2, 2, 1, n_extra=6)
        e.append(math.sqrt(O.l2_error_sq(h, u, W.sin_product_u)))
    r = e[1] / e[2]
    assert 3.4 < r < 4.4, e


def test_lshape_uniform_refinement_rate_four_thirds():
    """Sec. 5.2: uniform refinement of the L-shape converges like O(h^(4/3)) in L2."""
    e = _errors("lshape_l7", [4, 5, 6, 7])
    r = e[:-1] / e[1:]
    assert abs(r[-1] - 2 ** (4.0 / 3.0)) < 0.2, r


# ---------------------------------------------------------------- estimator (Alg. 4, Sec. 4)

def test_local_estimates_sum_to_global_norm():
    h, f, g, _ = _hier("lshape_l7", 5)
    prob = O.Problem(h, f, g)
    u, ws, _ = O.fmg(prob, 2, 2, 1)
    est = O.estimate(h, u, ws, 1)
    e = u - ws[h.L - 1]
    glob = e @ (h.levels[h.L].M @ e)                 # global mass matrix, not the per-macro sums
    assert abs((est["eta_T"] ** 2).sum() - glob) < 1e-12 * glob
    assert abs(est["err_l"] ** 2 - glob) < 1e-12 * glob   # j=1: e~_{L-1} is the same vector


def test_estimator_effectivity_in_theorem_bounds_for_smooth_problem():
    """Sec. 5.3: for a smooth solution and nu=2 the global effectivity of eta_1 lies inside
    [C1, C2] of Theorem 4.1 with theta = 1/4 (eps = 0)."""
    h, f, g, ue = _hier("square_l4", 6)
    prob = O.Problem(h, f, g)
    u, ws, _ = O.fmg(prob, 2, 2, 1)
    est = O.estimate(h, u, ws, 1)
    eff = est["eta_j"] / math.sqrt(O.l2_error_sq(h, u, ue))
    c1, c2 = O.theorem41_constants(0.25, 1)
    assert c1 <= eff <= c2, eff
    assert abs(est["theta"] - 0.25) < 0.05


def test_theorem41_constants_match_printed_tables():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "theorem41_constants.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for qn, qd, j, c1, c2 in rows:
        theta = 2.0 ** (-float(qn) / float(qd))
        got = O.theorem41_constants(theta, int(j))
        assert round(got[0], 2) == float(c1) and round(got[1], 2) == float(c2), (qn, qd, j, got)


def test_theorem41_limits():
    # eps = 0: both constants tend to one as j grows; eps > 0 widens them
    c1, c2 = O.theorem41_constants(0.25, 40)
    assert abs(c1 - 1) < 1e-9 and abs(c2 - 1) < 1e-9
    a1, a2 = O.theorem41_constants(0.25, 2, 0.1)
    b1, b2 = O.theorem41_constants(0.25, 2, 0.0)
    assert a1 < b1 and a2 > b2


def test_corollary_bounds_reduce_to_theorem_ratio():
    # Cor. 4.3 with theta_min = theta_max is C2/C1 of Theorem 4.1
    t = 0.25
    for j in (1, 2, 3):
        c1, c2 = O.theorem41_constants(t, j)
        s, _ = O.corollary_dgamma_bounds(t, t, j)
        assert abs(s - c2 / c1) < 1e-12 * s


# ---------------------------------------------------------------- marking (Sec. 5.1)

def test_marking_brute_force():
    rng = np.random.default_rng(7)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        eta = rng.random(n)
        if trial % 3 == 0:       # planted exact ties
            eta[rng.integers(0, n, size=n // 2)] = eta[0]
        frac = float(rng.choice([0.1, 0.2, 0.125, 0.5, 1.0 / 3.0]))
        got = O.mark_top_fraction(eta, frac)
        k = max(1, math.ceil(frac * n - 1e-9))
        kth = sorted(eta, reverse=True)[k - 1]
        assert got.sum() >= k
        assert set(np.nonzero(got)[0]) == {i for i in range(n) if eta[i] >= kth * (1 - 1e-8)}


def test_marking_count_is_not_fooled_by_rounding():
    # 0.1 * 30 = 3.0000000000000004 in floating point: three elements, not four
    assert O.mark_top_fraction(np.arange(30.0), 0.1).sum() == 3
