"""Oracle pins for 2D red-green refinement (Sec. 3), the adjoint gradients, and planted mistakes.

The red-green pins check geometric invariants (conformity, area, orientation, angle bounds),
not a stored copy of the oracle's output.  The adjoint is pinned by central finite differences
of exact sparse solves.  The planted-mistake tests break one piece of the oracle on purpose
(monkeypatched, CPU only) and assert that a pin above then fails.
"""

import math

import numpy as np
import pytest

import workloads as W
from oracle import hhg_oracle as O


def _edges(cells):
    cnt = {}
    for t in cells:
        for e in range(3):
            a, b = int(t[e]), int(t[(e + 1) % 3])
            key = (min(a, b), max(a, b))
            cnt[key] = cnt.get(key, 0) + 1
    return cnt


def _signed_area(co, t):
    a, b, c = co[t[0]], co[t[1]], co[t[2]]
    return 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))


def _on_lshape_boundary(p, q):
    """Both endpoints on one straight piece of the L-shape boundary."""
    for ax, val in ((0, -1.0), (0, 1.0), (1, -1.0), (1, 1.0)):
        if abs(p[ax] - val) < 1e-12 and abs(q[ax] - val) < 1e-12:
            return True
    if abs(p[1]) < 1e-12 and abs(q[1]) < 1e-12 and p[0] >= -1e-12 and q[0] >= -1e-12:
        return True
    if abs(p[0]) < 1e-12 and abs(q[0]) < 1e-12 and p[1] <= 1e-12 and q[1] <= 1e-12:
        return True
    return False


def _green_angle_bound(co, cells):
    best = _min_angle(co, cells)
    for t in cells:
        for e in range(3):
            a, b, c = t[(e + 2) % 3], t[e], t[(e + 1) % 3]
            m = 0.5 * (co[b] + co[c])
            pts = np.vstack([co, m])
            mi = len(co)
            best = min(best, _min_angle(pts, [(a, b, mi), (a, mi, c)]))
    return best


def _min_angle(co, cells):
    best = math.pi
    for t in cells:
        P = [np.array(co[v]) for v in t]
        for i in range(3):
            u = P[(i + 1) % 3] - P[i]
            v = P[(i + 2) % 3] - P[i]
            c = np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v))
            best = min(best, math.acos(max(-1.0, min(1.0, c))))
    return best


def test_rg2d_conforming_area_orientation_over_steps():
    co, ce = W.lshape_mesh()
    rg = O.RG2D(co, ce)
    rng = np.random.default_rng(11)
    # red children are similar to their parent and greens are reverted before each step, so
    # every triangle is similar to an initial one or is one green half of such a triangle
    a0 = _green_angle_bound(co, ce)
    for step in range(5):
        c, t = rg.mesh()
        marked = np.zeros(len(t), dtype=bool)
        marked[rng.choice(len(t), size=max(1, len(t) // 5), replace=False)] = True
        rg.refine(marked)
        c, t = rg.mesh()
        areas = np.array([_signed_area(c, x) for x in t])
        assert (areas > 0).all()
        assert abs(areas.sum() - 3.0) < 1e-12
        for (a, b), n in _edges(t).items():
            assert n in (1, 2)
            if n == 1:   # an unpaired edge must be on the domain boundary (no hanging nodes)
                assert _on_lshape_boundary(c[a], c[b]), (step, a, b)
        assert len(np.unique(t.ravel())) == len(c)      # every vertex is used
        assert _min_angle(c, t) >= a0 - 1e-12


def test_rg2d_marked_triangles_are_red_refined():
    co, ce = W.square_mesh(2)
    rg = O.RG2D(co, ce)
    marked = np.zeros(len(ce), dtype=bool)
    marked[[0, 5]] = True
    rg.refine(marked)
    c, t = rg.mesh()
    tris = {tuple(sorted(x)) for x in t.tolist()}
    for i in (0, 5):
        assert tuple(sorted(ce[i])) not in tris
        area = _signed_area(co, ce[i])
        # all four red children (area/4, inside the parent) are present
        kids = [x for x in t if abs(_signed_area(c, x) - area / 4) < 1e-14
                and all(_inside(c[v], co[ce[i]]) for v in x)]
        assert len(kids) == 4
    # unmarked triangles far from the marked ones survive unchanged
    assert len(t) > len(ce)


def _inside(p, tri):
    a, b, c = tri
    def s(p1, p2, p3):
        return (p1[0] - p3[0]) * (p2[1] - p3[1]) - (p2[0] - p3[0]) * (p1[1] - p3[1])
    d1, d2, d3 = s(p, a, b), s(p, b, c), s(p, c, a)
    neg = (d1 < -1e-14) or (d2 < -1e-14) or (d3 < -1e-14)
    pos = (d1 > 1e-14) or (d2 > 1e-14) or (d3 > 1e-14)
    return not (neg and pos)


def test_rg2d_marking_a_green_refines_its_parent():
    co, ce = W.square_mesh(2)
    rg = O.RG2D(co, ce)
    m = np.zeros(len(ce), dtype=bool)
    m[0] = True
    rg.refine(m)
    greens = [i for i, x in enumerate(rg.tris) if x[3] is not None]
    assert greens
    parent = rg.tris[greens[0]][3]
    m2 = np.zeros(len(rg.tris), dtype=bool)
    m2[greens[0]] = True
    rg.refine(m2)
    c, t = rg.mesh()
    tris = {tuple(sorted(x)) for x in t.tolist()}
    assert tuple(sorted(parent)) not in tris
    # the parent's centroid is now covered by red children of area parent/4
    pa = _signed_area(c, parent)
    cen = np.mean([c[v] for v in parent], axis=0)
    cover = [x for x in t if _inside(cen, [c[v] for v in x])]
    assert cover and all(abs(_signed_area(c, x) - pa / 4) < 1e-14 for x in cover)


# ---------------------------------------------------------------- adjoint

@pytest.mark.parametrize("name,L", [("fichera336_l6", 1), ("square_l4", 3)])
def test_adjoint_gradients_match_central_differences(name, L):
    co, ce, _, f, g, k, _ = W.workload(name, L)
    if k is None:
        k = W.coeff_uniform(len(ce), seed=5)
    centroid = co[ce].mean(axis=1)
    in_S = np.all(centroid > 0.5, axis=1)
    h = O.Hierarchy(co, ce, L, k=k)
    fL = f(h.levels[L].x) + 0.1 * np.sin(3 * h.levels[L].x.sum(axis=1))
    prob = O.Problem(h, fL, g)
    u = O.exact_solve(prob)
    J, gf, gk, _ = O.adjoint_gradients(h, u, in_S)

    def J_of(kk, ff):
        hh = O.Hierarchy(co, ce, L, k=kk)
        pp = O.Problem(hh, ff, g)
        uu = O.exact_solve(pp)
        return float(O.local_mass_sq(hh.levels[L], uu, len(ce))[in_S].sum())

    assert abs(J_of(k, fL) - J) < 1e-13 * J
    rng = np.random.default_rng(2)
    for t in rng.choice(len(ce), size=3, replace=False):
        eps = 1e-5 * k[t]
        kp, km = k.copy(), k.copy()
        kp[t] += eps
        km[t] -= eps
        fd = (J_of(kp, fL) - J_of(km, fL)) / (2 * eps)
        assert abs(fd - gk[t]) <= 1e-6 * max(abs(gk).max(), 1e-30), (t, fd, gk[t])
    free = np.nonzero(h.levels[L].free)[0]
    for j in rng.choice(free, size=3, replace=False):
        eps = 1e-4
        fp, fm = fL.copy(), fL.copy()
        fp[j] += eps
        fm[j] -= eps
        fd = (J_of(k, fp) - J_of(k, fm)) / (2 * eps)
        assert abs(fd - gf[j]) <= 1e-6 * abs(gf).max(), (j, fd, gf[j])


@pytest.mark.parametrize("name,L", [("fichera336_l6", 1), ("square_l4", 3)])
def test_adjoint_taylor_remainders(name, L):
    """Taylor test of the adjoint gradients along random directions.  The discrete solution is
    affine in the nodal source f, so J(f + e d) - J(f) - e <dJ/df, d> equals e^2 J(S d) exactly,
    where S d solves the problem with source d and zero boundary data (this also covers f at
    Dirichlet nodes, which reaches free rows through b = M f).  In k the remainder
    J(k + e dk) - J(k) - e <dJ/dk, dk> is O(e^2): it falls by a factor 4 when e is halved, where a
    wrong gradient leaves an O(e) remainder that falls by 2."""
    co, ce, _, f, g, k, _ = W.workload(name, L)
    if k is None:
        k = W.coeff_uniform(len(ce), seed=5)
    in_S = np.all(co[ce].mean(axis=1) > 0.5, axis=1)
    h = O.Hierarchy(co, ce, L, k=k)
    x = h.levels[L].x
    fL = f(x) + 0.1 * np.sin(3 * x.sum(axis=1))

    def J_of(hh, ff, gg):
        uu = O.exact_solve(O.Problem(hh, ff, gg))
        return float(O.local_mass_sq(hh.levels[L], uu, len(ce))[in_S].sum())

    def zero(y):
        return np.zeros(len(y))

    u = O.exact_solve(O.Problem(h, fL, g))
    J, gf, gk, _ = O.adjoint_gradients(h, u, in_S)
    rng = np.random.default_rng(7)
    d = rng.uniform(-1.0, 1.0, len(x))
    Jd = J_of(h, d, zero)
    assert Jd > 0
    for e in (1.0, 0.1):
        R = J_of(h, fL + e * d, g) - J - e * float(gf @ d)
        scale = max(J, e * abs(float(gf @ d)), e * e * Jd)
        assert abs(R - e * e * Jd) <= 1e-10 * scale, (e, R, e * e * Jd)
    dk = k * rng.uniform(-1.0, 1.0, len(k))
    slope = float(gk @ dk)
    R = [J_of(O.Hierarchy(co, ce, L, k=k + e * dk), fL, g) - J - e * slope for e in (1e-2, 5e-3)]
    assert abs(R[0]) <= 1e-2 * abs(slope), (R, slope)
    assert 3.6 <= R[0] / R[1] <= 4.4, R


# ---------------------------------------------------------------- planted mistakes

def test_planted_mass_mistake_is_caught(monkeypatch):
    real = O._element_matrices

    def wrong(X):
        K, M, vol = real(X)
        d = X.shape[2]
        return K, vol[:, None, None] * np.ones_like(M) / ((d + 1) * (d + 2)), vol  # dropped delta_ab
    monkeypatch.setattr(O, "_element_matrices", wrong)
    co, ce = W.square_mesh(2)
    h = O.Hierarchy(co, ce, 1)
    assert abs(h.levels[1].M.sum() - 1.0) > 1e-3


def test_planted_refinement_mistake_is_caught(monkeypatch):
    from test_oracle_pins import test_bey_refinement_is_the_kuhn_lattice as lattice_pin
    edges, children = O._bey_children_3d()
    bad = list(children)
    bad[4] = (4, 5, 6, 9)    # one child of the interior octahedron built on the wrong diagonal
    monkeypatch.setattr(O, "_bey_children_3d", lambda: (edges, bad))
    with pytest.raises(AssertionError):
        lattice_pin()


def test_planted_interpolation_weight_mistake_is_caught():
    co, ce = W.square_mesh(2)
    h = O.Hierarchy(co, ce, 2)
    P = h.levels[2].P.copy()
    P.data[P.data == 0.5] = 0.6
    xc, xf = h.levels[1].x, h.levels[2].x
    assert np.abs(P @ xc[:, 0] - xf[:, 0]).max() > 1e-3


def test_planted_estimator_sign_mistake_is_caught(monkeypatch):
    co, ce = W.lshape_mesh()
    L = 3
    h = O.Hierarchy(co, ce, L)
    g = lambda x: 1.0 + x[:, 0]
    prob = O.Problem(h, lambda x: np.zeros(len(x)), g)
    u, ws, _ = O.fmg(prob, 2, 2, 1)
    real = O.local_mass_sq
    monkeypatch.setattr(O, "prolong_to_finest", lambda hh, v, l: -_prolong(hh, v, l))
    est = O.estimate(h, u, ws, 1)
    assert est["err_l"] > 1e-3    # the linear-solution pin (estimate vanishes) would fail


def _prolong(h, v, l):
    for m in range(l + 1, h.L + 1):
        v = h.levels[m].P @ v
    return v
