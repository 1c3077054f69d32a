"""Pins of the estimator's alternative norms (Remark in Sec. 4) in the oracle: the energy form
against closed forms, the goal-oriented weighted seminorm against the L2 estimator, and the
convergence factor each norm measures."""

import math

import numpy as np
import pytest

import workloads as W
from oracle import hhg_oracle as O


def _areas(co, ce):
    X = co[ce]
    if co.shape[1] == 2:
        d1, d2 = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
        return np.abs(d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]) / 2
    return np.abs(np.einsum("ij,ij->i", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0])) / 6


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_form_of_a_linear_function(dim):
    """int_T k_T |grad e|^2 = k_T |a|^2 |T| for e = a.x + c, with a random coefficient per cell."""
    co, ce = W.square_mesh(2) if dim == 2 else W.cube_mesh(1)
    rng = np.random.default_rng(11)
    k = rng.uniform(0.5, 3.0, len(ce))
    h = O.Hierarchy(co, ce, 2, k=k)
    a = np.array([0.7, -1.3, 0.4][:dim])
    lev = h.levels[2]
    e = lev.x @ a + 0.25
    got = O.local_energy_sq(lev, e, len(ce))
    want = k * (a @ a) * _areas(co, ce)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_energy_form_of_the_interpolant_of_x_squared(L):
    """On the unit square (4 x 2 right triangles, every micro triangle spanning one x-strip of width
    h with its vertices on the strip's edges) the interpolant of x^2 has slope 2a + h on the strip
    [a, a + h], so int |grad I x^2|^2 = h^3 sum_m (2m + 1)^2 = h^3 n (4 n^2 - 1) / 3, n = 1/h."""
    co, ce = W.square_mesh(2)
    h = O.Hierarchy(co, ce, L)
    lev = h.levels[L]
    n = 2 * 2 ** L
    hh = 1.0 / n
    total = O.local_energy_sq(lev, lev.x[:, 0] ** 2, len(ce)).sum()
    assert abs(total - hh ** 3 * n * (4 * n * n - 1) / 3) < 1e-13


def _solved(L=5):
    co, ce = W.square_mesh(2)
    h = O.Hierarchy(co, ce, L)
    u, ws, _ = O.fmg(O.Problem(h, W.sin_product_f, W.sin_product_u), 2, 2, 2)
    return h, u, ws


def test_goal_seminorm_with_unit_weights_is_the_l2_estimator():
    h, u, ws = _solved()
    a = O.estimate(h, u, ws, 2)
    b = O.estimate(h, u, ws, 2, norm="goal", weights=np.ones(h.n_cells))
    for key in ("eta_j", "theta", "err_l", "err_lm1"):
        assert a[key] == pytest.approx(b[key], rel=1e-15)
    assert np.array_equal(a["eta_T"], b["eta_T"])


def test_goal_seminorm_on_a_subregion():
    """Indicator weights of a subset S of the macro cells: local indicators vanish outside S, equal
    the L2 ones inside, and the global values are the L2 sums over S alone."""
    h, u, ws = _solved()
    S = np.zeros(h.n_cells)
    S[[0, 3, 5]] = 1.0
    a = O.estimate(h, u, ws, 1)
    g = O.estimate(h, u, ws, 1, norm="goal", weights=S)
    assert np.all(g["eta_T"][S == 0] == 0)
    assert np.array_equal(g["eta_T"][S == 1], a["eta_T"][S == 1])
    err_l = math.sqrt(a["sq_l_T"][S == 1].sum())
    err_lm1 = math.sqrt(a["sq_lm1_T"][S == 1].sum())
    assert g["err_l"] == pytest.approx(err_l, rel=1e-14)
    assert g["eta_j"] == pytest.approx(err_l ** 2 / err_lm1, rel=1e-14)


def test_energy_estimator_vanishes_for_a_linear_solution():
    co, ce = W.square_mesh(2)
    h = O.Hierarchy(co, ce, 4)
    lin = lambda x: 1.0 + 0.5 * x[:, 0] - 2.0 * x[:, 1]
    u, ws, _ = O.fmg(O.Problem(h, lambda x: np.zeros(len(x)), lin), 2, 2, 2, 20)
    est = O.estimate(h, u, ws, 1, norm="energy")
    assert est["err_l"] < 1e-12 and np.abs(est["eta_T"]).max() < 1e-12


def test_convergence_factor_of_each_norm():
    """Smooth solution on uniform refinements, errors e_l ~ C theta^l with theta = 2^-2 in L2 and
    2^-1 in the energy norm.  In L2 the differences of successive solutions scale like the errors:
    theta~ = ||u_L - w_{L-1}|| / ||u_L - w_{L-2}|| -> (1/theta - 1) / (1/theta^2 - 1) = 3/15.  In the
    energy norm Galerkin orthogonality gives ||u_L - u_l||^2 = ||u - u_l||^2 - ||u - u_L||^2, so
    theta~^2 -> (1/theta^2 - 1) / (1/theta^4 - 1) = 3/15 and theta~ -> 1/sqrt(5)."""
    h, u, ws = _solved(L=6)
    th_l2 = O.estimate(h, u, ws, 1)["theta"]
    th_en = O.estimate(h, u, ws, 1, norm="energy")["theta"]
    assert abs(th_l2 - 3 / 15) < 0.005
    assert abs(th_en - 1 / math.sqrt(5)) < 1e-3


def test_unknown_norm_is_rejected():
    h, u, ws = _solved(L=3)
    with pytest.raises(ValueError):
        O.estimate(h, u, ws, 1, norm="h2")
