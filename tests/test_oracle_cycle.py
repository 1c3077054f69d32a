"""Pins of the oracle's V-cycle and FMG composition (Alg. 4) by linear algebra, not by convergence.

With a zero right-hand side and zero Dirichlet values a V(pre, post)-cycle maps the error e of the
free nodes linearly.  On two levels, with the exact coarse solve, that map is

    V_1 = S^post (I - P A_0^{-1} P^T A) S^pre,

and on three levels the coarse problem is solved by one V-cycle from zero, so its solution is
(I - V_1) A_1^{-1} times the restricted residual:

    V_2 = S^post (I - P_2 (I - V_1) A_1^{-1} P_2^T A_2) S^pre.

S (one smoothing sweep with zero right-hand side) is built column by column from the pinned `smooth`,
A_l^{-1} by a dense numpy solve, P from the pinned interpolation.  These matrices fix the number of
pre- and post-smoothing sweeps, their order around the coarse correction, the sign of the correction
and the recursion; a contraction bound alone would miss each of those mistakes.  FMG is pinned by
its call sequence: nu V-cycles on every level 0..L in order, n_extra more on level L, each level's
first V-cycle starting from the interpolated coarse iterate with the Dirichlet values of g, and
w_l being exactly that starting vector.
"""

import numpy as np
import pytest

import workloads as W
from oracle import hhg_oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _cases():
    co3, ce3 = W.perturbed_mesh("cube", seed=2)
    return {
        # 2D: 8 triangles, 1 free macro vertex, 2 levels below the top
        "square": (*W.square_mesh(2), None),
        # 2D general triangles (7-point stencils, 3 interior colours)
        "lshape_pert": (*W.perturbed_mesh("lshape"), None),
        # 3D general tets with per-cell coefficients (face block, 15-point stencils)
        "cube_pert_k": (co3, ce3, W.coeff_uniform(len(ce3), seed=3)),
    }


def _problem(name, L):
    co, ce, k = _cases()[name]
    h = O.Hierarchy(co, ce, L, k=k)
    zero = lambda x: np.zeros(len(x))
    return h, O.Problem(h, zero, zero)


def _smoother_matrix(lev):
    """S on the free nodes: column i is one sweep applied to the unit error e_i (rhs = 0)."""
    F = np.nonzero(lev.free)[0]
    S = np.zeros((len(F), len(F)))
    zero = np.zeros(len(lev.keys))
    for c, i in enumerate(F):
        u = np.zeros(len(lev.keys))
        u[i] = 1.0
        O.smooth(lev, u, zero)
        assert np.all(u[lev.dirichlet] == 0.0)
        S[:, c] = u[F]
    return S


def _free_blocks(h, l):
    lev = h.levels[l]
    F = np.nonzero(lev.free)[0]
    A = lev.A[F][:, F].toarray()
    P = None
    if l >= 1:
        Fc = np.nonzero(h.levels[l - 1].free)[0]
        P = lev.P[F][:, Fc].toarray()
    return F, A, P


def _vcycle_matrix(h, l, pre, post):
    """Error propagation of one V(pre, post)-cycle on level l (free nodes), built from the pinned
    pieces; level 0 is the exact solve (error propagation 0)."""
    F, A, P = _free_blocks(h, l)
    if l == 0:
        return np.zeros((len(F), len(F)))
    S = _smoother_matrix(h.levels[l])
    _, Ac, _ = _free_blocks(h, l - 1)
    Vc = _vcycle_matrix(h, l - 1, pre, post)
    # one V-cycle from zero on the coarse level solves A_c x = r to (I - V_c) A_c^{-1} r
    coarse = (np.eye(len(Ac)) - Vc) @ np.linalg.solve(Ac, np.eye(len(Ac))) if len(Ac) else np.zeros((0, 0))
    K = np.eye(len(F)) - P @ coarse @ P.T @ A
    return np.linalg.matrix_power(S, post) @ K @ np.linalg.matrix_power(S, pre)


@pytest.mark.parametrize("name,L", [("square", 2), ("lshape_pert", 2), ("cube_pert_k", 2)])
@pytest.mark.parametrize("pre,post", [(2, 1), (1, 2), (0, 1), (3, 0)])
def test_vcycle_is_the_composed_error_propagation(name, L, pre, post):
    h, prob = _problem(name, L)
    rng = np.random.default_rng(7)
    for l in range(1, L + 1):
        lev = h.levels[l]
        F = np.nonzero(lev.free)[0]
        V = _vcycle_matrix(h, l, pre, post)
        for _ in range(2):
            e = np.zeros(len(lev.keys))
            e[F] = rng.standard_normal(len(F))
            u = e.copy()
            O.vcycle(prob, l, u, np.zeros(len(lev.keys)), pre, post)
            assert np.all(u[lev.dirichlet] == 0.0)
            ref = V @ e[F]
            assert np.abs(u[F] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (l, pre, post)


def test_swapped_sweep_counts_or_flipped_correction_are_detected():
    """The composed matrix separates the readings a convergence test cannot: V(2,1) differs from
    V(1,2) and from the cycle with the coarse correction subtracted."""
    h, prob = _problem("cube_pert_k", 1)
    lev = h.levels[1]
    F = np.nonzero(lev.free)[0]
    V21 = _vcycle_matrix(h, 1, 2, 1)
    V12 = _vcycle_matrix(h, 1, 1, 2)
    S = _smoother_matrix(lev)
    _, A, P = _free_blocks(h, 1)
    _, A0, _ = _free_blocks(h, 0)
    Kflip = np.eye(len(F)) + P @ np.linalg.solve(A0, P.T @ A)
    Vflip = S @ Kflip @ S @ S
    e = np.zeros(len(lev.keys))
    e[F] = np.random.default_rng(3).standard_normal(len(F))
    u = e.copy()
    O.vcycle(prob, 1, u, np.zeros(len(lev.keys)), 2, 1)
    got = u[F]
    assert np.abs(got - V21 @ e[F]).max() < 1e-12 * np.abs(got).max()
    assert np.abs(got - V12 @ e[F]).max() > 1e-6 * np.abs(got).max()
    assert np.abs(got - Vflip @ e[F]).max() > 1e-6 * np.abs(got).max()


@pytest.mark.parametrize("nu,pre,post,n_extra", [(2, 2, 1, 0), (1, 1, 2, 3), (3, 2, 2, 1)])
def test_fmg_call_sequence_and_stored_iterates(monkeypatch, nu, pre, post, n_extra):
    co, ce, k = _cases()["cube_pert_k"]
    L = 2
    h = O.Hierarchy(co, ce, L, k=k)
    f = lambda x: np.sin(3 * x[:, 0]) + x[:, 1] * x[:, 2]
    g = lambda x: 0.5 + x[:, 0] - x[:, 1] * x[:, 2]
    prob = O.Problem(h, f, g)
    calls = []
    depth = [0]
    inner = O.vcycle

    def spy(prob_, l, u, rhs, pre_=2, post_=1):
        if depth[0] == 0:  # a call from fmg itself, not the V-cycle's own recursion
            calls.append((l, u.copy(), rhs is prob_.b[l], pre_, post_))
        depth[0] += 1
        try:
            inner(prob_, l, u, rhs, pre_, post_)
        finally:
            depth[0] -= 1

    monkeypatch.setattr(O, "vcycle", spy)
    uL, ws, us = O.fmg(prob, nu, pre, post, n_extra)
    levels = [c[0] for c in calls]
    assert levels == [l for l in range(L + 1) for _ in range(nu)] + [L] * n_extra
    assert all(c[2] and c[3] == pre and c[4] == post for c in calls)
    # level 0 starts from g on Dirichlet nodes, 0 elsewhere
    lev0 = h.levels[0]
    assert np.array_equal(calls[0][1], np.where(lev0.dirichlet, prob.g[0], 0.0))
    for l in range(L):
        fine = h.levels[l + 1]
        start = calls[(l + 1) * nu][1]               # before the first level-(l+1) V-cycle
        expect = fine.P @ us[l]
        expect[fine.dirichlet] = prob.g[l + 1][fine.dirichlet]
        assert np.array_equal(start, expect)
        assert np.array_equal(ws[l], start)           # w_l is the interpolated iterate
    # us[l] is the iterate after level l's nu V-cycles; u_L after the extra cycles as well
    monkeypatch.setattr(O, "vcycle", inner)
    u_ref = np.where(lev0.dirichlet, prob.g[0], 0.0)
    for l in range(L + 1):
        for _ in range(nu):
            O.vcycle(prob, l, u_ref, prob.b[l], pre, post)
        assert np.array_equal(u_ref, us[l])
        if l < L:
            u_ref = h.levels[l + 1].P @ u_ref
            u_ref[h.levels[l + 1].dirichlet] = prob.g[l + 1][h.levels[l + 1].dirichlet]
    for _ in range(n_extra):
        O.vcycle(prob, L, u_ref, prob.b[L], pre, post)
    assert np.array_equal(u_ref, uL)


def _colour_stage_sweep(lev, u, rhs):
    """The colour-stage reading of the sweep: every stage (the three face colours included) Jacobi
    inside the stage, in the oracle's stage order, with current values of everything else."""
    for s in range(len(lev.stages)):
        idx = lev.stages[s]
        if len(idx):
            u[idx] += (rhs[idx] - lev.stage_rows[s] @ u) / lev.stage_diag[s]


def _contraction(h, prob, L, cycles=30):
    lev = h.levels[L]
    e = np.where(lev.free, np.random.default_rng(0).standard_normal(len(lev.keys)), 0.0)
    zero = np.zeros(len(lev.keys))
    norms = []
    for _ in range(cycles + 1):
        norms.append(float(np.sqrt(e @ (lev.A @ e))))
        O.vcycle(prob, L, e, zero, 2, 1)
    return (norms[-1] / norms[-6]) ** (1 / 5)


def test_face_block_contracts_like_colour_stages(monkeypatch):
    """The face block (every macro face Gauss-Seidel on its own, surroundings frozen at the block
    start) against the colour-stage reading of the face stages: asymptotic V(2,1) contraction on a
    perturbed variable-k cube at L = 3, within 5 % of each other."""
    h, prob = _problem("cube_pert_k", 3)
    r_block = _contraction(h, prob, 3)
    monkeypatch.setattr(O, "smooth", _colour_stage_sweep)
    r_stage = _contraction(h, prob, 3)
    assert 0.05 < r_block < 0.5 and 0.05 < r_stage < 0.5
    assert abs(r_block - r_stage) <= 0.05 * r_stage, (r_block, r_stage)
