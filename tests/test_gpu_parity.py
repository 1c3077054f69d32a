"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerance: 1e-10 relative to the largest oracle value (binary64 results differ only by summation
order).  Marked sets must be identical.  Library nodes are matched to oracle nodes by coordinates.
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
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06049_gb300 as pkg
    pkg.lib()
    return pkg


def perturbed(name, seed=4, amp=0.12, m=2):
    return W.perturbed_mesh(name, seed=seed, amp=amp, m=m)


CASES = {
    "square": lambda: (*W.square_mesh(2), 4, None),
    "lshape": lambda: (*W.lshape_mesh(), 5, None),
    "lshape_pert": lambda: (*perturbed("lshape"), 4, None),
    "cube384": lambda: (*W.cube_mesh(4), 3, None),
    "cube_pert_k": lambda: (*perturbed("cube"), 3, W.coeff_uniform(48, seed=3)),
    # L = 3 is the first level of the 3072-tet cube whose face block takes the binary64 sparse
    # slot loop (macro faces x face-interior nodes >= 1e5: 6528 x 21), the path the full-size
    # binary64 solves take on their finest levels
    "cube3072_k": lambda: (*W.cube_mesh(8), 3, W.coeff_loguniform(3072, seed=0)),
    # general tets (15-point stencils, 4 interior colours) on the same sparse face path
    "cube3072_pert_k": lambda: (*perturbed("cube", seed=6, m=8), 3, W.coeff_loguniform(3072, seed=0)),
    "fichera_k": lambda: (*W.fichera_mesh(), 3, W.coeff_uniform(336, seed=1)),
}

_cache = {}


def setup_case(P, name):
    if name in _cache:
        return _cache[name]
    co, ce, L, k = CASES[name]()
    h = O.Hierarchy(co, ce, L, k=k)
    mesh = P.Mesh(co, ce, L)
    if k is not None:
        mesh.set_coefficient(k)
    maps = []
    for l in range(L + 1):
        x = mesh.level_coords(l)
        dist, idx = cKDTree(h.levels[l].x).query(x)
        assert dist.max() < 1e-9
        maps.append(idx)
    _cache[name] = (co, ce, L, k, h, mesh, maps)
    return _cache[name]


def fg(dim):
    if dim == 2:
        return (lambda x: np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]) + 1.0,
                lambda x: 0.25 + x[:, 0] * x[:, 1])
    return (lambda x: np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]) + x[:, 2],
            lambda x: 0.1 * x[:, 0] - x[:, 2] * x[:, 1])


def copy_sum(v, mp):
    """Sum of a per-copy vector over the copies of each node (mp: layout entry -> oracle node),
    written back to every copy."""
    return np.bincount(mp, weights=v, minlength=int(mp.max()) + 1)[mp]


def close(gpu, ref, tol=TOL):
    scale = max(np.abs(ref).max(), 1e-300)
    err = np.abs(gpu - ref).max() / scale
    assert err <= tol, err


def close_estimates(eg, eo, h, uo):
    """Estimator parity.  eta_T = ||u_L - w_{L-1}||_T is the norm of a difference of two FMG iterates
    (|e~| ~ 1e-5 |u|), so agreement of u_L and w to 1e-10 relative bounds eta_T only to
    1e-10 ||u_L||_T: the tolerance is 1e-10 relative to the norm of the solution over the same cell
    (and over the domain for the global values)."""
    u_T = np.sqrt(O.local_mass_sq(h.levels[h.L], uo, h.n_cells))
    assert np.all(np.abs(eg["eta_T"] - eo["eta_T"]) <= TOL * u_T)
    u_glob = math.sqrt(float((u_T ** 2).sum()))
    for key in ("err_l", "err_lm1"):
        assert abs(eg[key] - eo[key]) <= TOL * u_glob, key
    # theta and eta_j are ratios / products of those norms: first-order error propagation
    rel = TOL * u_glob * (1 / eo["err_l"] + 1 / eo["err_lm1"])
    assert abs(eg["theta"] - eo["theta"]) <= rel * eo["theta"]


def test_cases_reach_the_sparse_face_path():
    """The binary64 face block switches to its sparse slot loop when macro faces x face-interior
    nodes reach 1e5; the two 3072-tet cases are above that on their finest level (and below it on
    the level under it), so the parity tests below cover both loops."""
    for name in ("cube3072_k", "cube3072_pert_k"):
        co, ce, L, _ = CASES[name]()
        tri = np.sort(ce[:, [[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]]].reshape(-1, 3), axis=1)
        n_faces = len(np.unique(tri, axis=0))
        nf = lambda l: (2 ** l - 1) * (2 ** l - 2) // 2
        assert n_faces * nf(L) >= 100000 > n_faces * nf(L - 1), (name, n_faces)


@pytest.mark.parametrize("name", list(CASES))
def test_operators_match_assembled_matrices(P, name):
    co, ce, L, k, h, mesh, maps = setup_case(P, name)
    rng = np.random.default_rng(0)
    for l in range(L + 1):
        lev = h.levels[l]
        xo = rng.standard_normal(len(lev.keys))
        x = np.ascontiguousarray(xo[maps[l]])
        close(mesh.apply(l, 0, x), (lev.A @ xo)[maps[l]], 1e-12)
        close(mesh.apply(l, 1, x), (lev.M @ xo)[maps[l]], 1e-12)
        if l >= 1:
            xc = rng.standard_normal(len(h.levels[l - 1].keys))
            out = mesh.apply(l, 2, np.ascontiguousarray(xc[maps[l - 1]]))
            close(out, (lev.P @ xc)[maps[l]], 1e-13)


@pytest.mark.parametrize("name", list(CASES))
def test_smoothing_sweeps_match(P, name):
    co, ce, L, k, h, mesh, maps = setup_case(P, name)
    rng = np.random.default_rng(1)
    for l in range(1, L + 1):
        lev = h.levels[l]
        fo = rng.standard_normal(len(lev.keys))
        u0 = np.where(lev.dirichlet, rng.standard_normal(len(lev.keys)), rng.standard_normal(len(lev.keys)))
        for ns in (1, 3):
            uo = u0.copy()
            for _ in range(ns):
                O.smooth(lev, uo, lev.M @ fo)
            ug = np.ascontiguousarray(u0[maps[l]])
            mesh.apply(l, 3, np.ascontiguousarray(fo[maps[l]]), ug, nsweeps=ns)
            close(ug, uo[maps[l]])


def run_both(P, name, nu=2, pre=2, post=1, n_extra=0):
    co, ce, L, k, h, mesh, maps = setup_case(P, name)
    f, g = fg(h.dim)
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    u = mesh.solve(nu=nu, pre=pre, post=post, n_extra=n_extra)
    prob = O.Problem(h, f, g)
    uo, ws, _ = O.fmg(prob, nu, pre, post, n_extra)
    return mesh, maps, h, u, uo, ws


@pytest.mark.parametrize("name", list(CASES))
def test_fmg_solution_and_stored_coarse_solutions(P, name):
    mesh, maps, h, u, uo, ws = run_both(P, name)
    close(u, uo[maps[h.L]])
    for l in range(h.L):
        close(mesh.get_vector(1, l), ws[l][maps[l + 1]])


@pytest.mark.parametrize("name", ["lshape_pert", "cube_pert_k", "fichera_k", "cube3072_k"])
def test_fmg_with_restricted_coarse_rhs(P, name):
    """rhs = 1: b_L = M_L f_L and b_l = I^T b_{l+1} on the coarser levels (the oracle's
    Problem(rhs="restricted")): every level's right-hand side on the free nodes, u_L and every stored
    w_l against the oracle, and (on the meshes whose exact discrete solution the oracle's sparse
    direct solve finds in seconds) the mixed solve's refinement to that solution."""
    co, ce, L, k, h, mesh, maps = setup_case(P, name)
    f, g = fg(h.dim)
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    u = mesh.solve(nu=2, pre=2, post=1, rhs=1)
    prob = O.Problem(h, f, g, rhs="restricted")
    for l in range(L + 1):
        free = h.levels[l].free[maps[l]]
        close(mesh.get_vector(2, l)[free], prob.b[l][maps[l]][free])
    uo, ws, _ = O.fmg(prob, 2, 2, 1)
    close(u, uo[maps[L]])
    for l in range(L):
        close(mesh.get_vector(1, l), ws[l][maps[l + 1]])
    if len(h.levels[L].keys) <= 100000:
        um = mesh.solve(nu=2, pre=2, post=1, precision=1, storage=0, ir_steps=12, ir_vcycles=2, rhs=1)
        ex = O.exact_solve(prob)
        close(um, ex[maps[L]])


@pytest.mark.parametrize("name,nu,pre,post,extra", [("lshape", 1, 1, 1, 2), ("cube384", 3, 1, 2, 1),
                                                     ("fichera_k", 1, 2, 2, 0)])
def test_fmg_other_cycle_parameters(P, name, nu, pre, post, extra):
    mesh, maps, h, u, uo, ws = run_both(P, name, nu, pre, post, extra)
    close(u, uo[maps[h.L]])


@pytest.mark.parametrize("name", list(CASES))
def test_estimator_and_marking(P, name):
    mesh, maps, h, u, uo, ws = run_both(P, name)
    for j in range(1, h.L):
        eg = mesh.estimate(j)
        eo = O.estimate(h, uo, ws, j)
        close_estimates(eg, eo, h, uo)
        assert abs(eg["err_Lm1"] ** 2 - (eo["eta_T"] ** 2).sum()) <= 1e-10 * eg["err_Lm1"] ** 2
        for frac in (0.1, 0.2, 0.125):
            assert np.array_equal(P.mark(eg["eta_T"], frac), O.mark_top_fraction(eo["eta_T"], frac))


@pytest.mark.parametrize("name", list(CASES))
def test_estimator_in_other_norms(P, name):
    """The energy norm and the per-cell weighted L2 seminorm of the Remark in Sec. 4 against the
    oracle.  Energy: u_L and the w_l agree to 1e-10 max|u| node by node (the FMG parity test), so
    each difference vector agrees to twice that, and the seminorm of a nodal vector d on T is at most
    max|d| sqrt(sum_pq |A_T,pq|): per-cell tolerance 1e-10 * 2 max|u| sqrt(sum |A_T|).  Weighted:
    1e-10 sqrt(w_T) ||u||_{L2,T}, exact zeros where w_T = 0; norm 0 through the same entry point
    gives hhg_estimate's values bit for bit."""
    mesh, maps, h, u, uo, ws = run_both(P, name)
    levL = h.levels[h.L]
    uM = np.sqrt(O.local_mass_sq(levL, uo, h.n_cells))
    absA_T = np.bincount(levL.emacro, weights=np.abs(levL.Ke).sum(axis=(1, 2)), minlength=h.n_cells)
    sE_T = 2 * np.abs(uo).max() * np.sqrt(absA_T)
    sE = math.sqrt(float((sE_T ** 2).sum()))
    rng = np.random.default_rng(5)
    w = rng.uniform(0, 2, h.n_cells)
    w[::3] = 0.0
    sW_T = np.sqrt(w) * uM
    sW = math.sqrt(float((sW_T ** 2).sum()))
    for j in range(1, h.L):
        a = mesh.estimate(j)
        b = mesh.estimate(j, norm=0, weights=np.ones(h.n_cells))
        assert np.array_equal(a["eta_T"], b["eta_T"]) and a["eta_j"] == b["eta_j"]
        for norm, key, s_T, s in ((1, "energy", sE_T, sE), (2, "goal", sW_T, sW)):
            eg = mesh.estimate(j, norm=norm, weights=w if norm == 2 else None)
            eo = O.estimate(h, uo, ws, j, norm=key, weights=w if norm == 2 else None)
            assert np.all(np.abs(eg["eta_T"] - eo["eta_T"]) <= TOL * s_T), key
            # eta_jT = theta_T^j ||e~_l||_T: first-order propagation of the per-cell norm errors
            with np.errstate(divide="ignore", invalid="ignore"):
                inv = 1 / np.sqrt(eo["sq_l_T"]) + 1 / np.sqrt(eo["sq_lm1_T"])
                tol_jT = np.where(np.isfinite(inv), 4 * (j + 1) * TOL * s_T * inv * eo["eta_jT"], np.inf)
            assert np.all(np.abs(eg["eta_jT"] - eo["eta_jT"]) <= tol_jT + 1e-300), key
            for k in ("err_l", "err_lm1"):
                assert abs(eg[k] - eo[k]) <= TOL * s, (key, k)
            rel = TOL * s * (1 / eo["err_l"] + 1 / eo["err_lm1"])
            assert abs(eg["theta"] - eo["theta"]) <= rel * eo["theta"], key
            if norm == 2:
                assert np.all(eg["eta_T"][w == 0] == 0)
    with pytest.raises(P.HHGError):
        mesh.estimate(1, norm=3)
    with pytest.raises(P.HHGError):
        mesh.estimate(1, norm=2, weights=-np.ones(h.n_cells))


def test_estimate_before_solve_is_an_error(P):
    co, ce = W.square_mesh(2)
    m = P.Mesh(co, ce, 3)
    with pytest.raises(P.HHGError):
        m.estimate(1)
    with pytest.raises(P.HHGError):
        m.solve()  # no data yet
    m.close()


def test_invalid_inputs_are_rejected(P):
    co, ce = W.square_mesh(2)
    with pytest.raises(P.HHGError):
        P.Mesh(co, ce, 0)
    bad = ce.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(P.HHGError):
        P.Mesh(co, bad, 2)
    m = P.Mesh(co, ce, 2)
    with pytest.raises(P.HHGError):
        m.set_coefficient(-np.ones(len(ce)))
    x = m.level_coords(2)
    m.set_data(np.full(len(x), np.nan), np.zeros(len(x)))
    with pytest.raises(P.HHGError) as e:
        m.solve()
    assert e.value.status == 6  # HHG_ERR_DIVERGED
    m.close()


def test_device_tensors_and_streams(P):
    """Inputs/outputs as CUDA tensors on a user stream give the same result as host arrays."""
    import torch
    co, ce = W.lshape_mesh()
    L = 4
    s = torch.cuda.Stream()
    m1 = P.Mesh(co, ce, L)
    m2 = P.Mesh(co, ce, L, stream=s)
    x = m1.level_coords(L)
    f = np.ascontiguousarray(np.cos(x[:, 0]) + x[:, 1])
    g = np.ascontiguousarray(W.lshape_g(x))
    m1.set_data(f, g)
    u1 = m1.solve()
    with torch.cuda.stream(s):
        fd = torch.from_numpy(f).cuda()
        gd = torch.from_numpy(g).cuda()
        out = torch.empty_like(fd)
    m2.set_data(fd, gd)
    m2.solve(out=out)
    s.synchronize()
    assert np.array_equal(out.cpu().numpy(), u1)    # same kernels, same order: bitwise equal
    m1.close()
    m2.close()


@pytest.mark.parametrize("name", ["fichera_k", "square"])
def test_adjoint_gradients_match_oracle(P, name):
    co, ce, L, k, h, mesh, maps = setup_case(P, name)
    f, g = fg(h.dim)
    if name == "fichera_k":
        g = lambda x: np.zeros(len(x))
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    mesh.solve(nu=2, pre=2, post=1, n_extra=60)
    in_S = np.all(co[ce].mean(axis=1) > 0.5, axis=1)
    J, gf, gk = mesh.adjoint_l2(in_S, nu=2, pre=2, post=1, n_extra=60)
    prob = O.Problem(h, f, g)
    uo = O.exact_solve(prob)
    Jo, gfo, gko, _ = O.adjoint_gradients(h, uo, in_S)
    assert abs(J - Jo) <= 1e-9 * abs(Jo)
    close(copy_sum(gf, maps[L]), gfo[maps[L]], 1e-9)
    close(gk, gko, 1e-9)


def test_full_size_lshape_matches_oracle(P):
    """The L-shape at its full level L=7 (the oracle finishes in seconds)."""
    co, ce, L, f, g, k, _ = W.workload("lshape_l7")
    mesh = P.Mesh(co, ce, L)
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    u = mesh.solve()
    h = O.Hierarchy(co, ce, L)
    prob = O.Problem(h, f, g)
    uo, ws, _ = O.fmg(prob, 2, 2, 1)
    _, idx = cKDTree(h.levels[L].x).query(x)
    close(u, uo[idx])
    eg = mesh.estimate(1)
    eo = O.estimate(h, uo, ws, 1)
    close_estimates(eg, eo, h, uo)
    assert np.array_equal(P.mark(eg["eta_T"], 0.2), O.mark_top_fraction(eo["eta_T"], 0.2))
    mesh.close()


def test_full_size_cube384_l6_properties(P):
    """Full-size 3D workload (16.6 M unknowns): second-order convergence against the exact solution
    (ratio of the L2 errors at L=5 and L=6 near 4) and the estimator inside Theorem 4.1's bounds."""
    errs = []
    for L in (5, 6):
        co, ce, _, f, g, k, ue = W.workload("cube384_l6", L)
        mesh = P.Mesh(co, ce, L)
        x = mesh.level_coords(L)
        mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
        u = mesh.solve()
        e = np.ascontiguousarray(ue(x) - u)
        Me = mesh.apply(L, 1, e)
        # interface nodes appear once per adjacent cell: weight each copy by 1/multiplicity
        _, inv, cnt = np.unique(np.round(x * 2 ** (L + 3)).astype(np.int64), axis=0, return_inverse=True,
                                return_counts=True)
        wgt = 1.0 / cnt[inv.ravel()]
        errs.append(math.sqrt(np.sum(wgt * e * Me)))
        est = mesh.estimate(1)
        eff = est["eta_j"] / errs[-1]
        c1, c2 = O.theorem41_constants(0.25, 1)
        assert c1 <= eff <= c2, eff
        assert mesh.info.n_unknowns == (4 * 2 ** L - 1) ** 3
        mesh.close()
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_full_size_cube384_l6_sampled_estimator_parity(P):
    """The benchmark workload at its full size (384-tet cube, L = 6, 16.6 M unknowns; binary64 FMG
    with nu = 2, V(2,1) and 4 extra V-cycles, the solve and estimator graphs bench.py times).
    eta_T is local: eta_T^2 = (u_L - w_{L-1})^T M_{L,T} (u_L - w_{L-1}) over macro cell T's own
    closure nodes.  For sampled cells the oracle recomputes it from the library's u_L and w_{L-1} on
    that cell alone (a one-cell hierarchy, mass matrix assembled element by element); the squared
    indicators sum to ||e~_{L-1}||^2 and the marking equals the oracle's marking of them."""
    co, ce, L, f, g, k, _ = W.workload("cube384_l6")
    _sampled_estimator_parity(P, co, ce, L, f, g)


def _sampled_estimator_parity(P, co, ce, L, f, g, n_sample=4):
    mesh = P.Mesh(co, ce, L)
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    u = mesh.solve(nu=2, pre=2, post=1, n_extra=4)
    w = mesh.get_vector(1, L - 1)
    est = mesh.estimate(1)
    nc = len(ce)
    Nt = len(x) // nc
    assert Nt * nc == len(x)
    rng = np.random.default_rng(11)
    cells = sorted({0, nc - 1} | set(rng.choice(nc, n_sample, replace=False).tolist()))
    for T in cells:
        hT = O.Hierarchy(co[ce[T]], np.arange(co.shape[1] + 1)[None, :], L)
        lev = hT.levels[L]
        sl = slice(T * Nt, (T + 1) * Nt)
        dist, idx = cKDTree(x[sl]).query(lev.x)
        assert dist.max() < 1e-9 and len(np.unique(idx)) == Nt
        e = (u[sl] - w[sl])[idx]
        ref = float(e @ (lev.M @ e))
        assert abs(est["eta_T"][T] ** 2 - ref) <= TOL * ref, (T, est["eta_T"][T] ** 2, ref)
    sq = est["eta_T"] ** 2
    assert abs(est["err_Lm1"] ** 2 - sq.sum()) <= TOL * sq.sum()
    assert np.array_equal(P.mark(est["eta_T"], 0.125), O.mark_top_fraction(est["eta_T"], 0.125))
    mesh.close()


@pytest.mark.parametrize("name", ["lshape_pert", "cube_pert_k"])
def test_estimator_pair_form_against_binary64_forms(P, name):
    """hhg_estimate evaluates its per-cell L2 forms in binary32 hi/lo pairs.  Against the binary64
    form e^T M_T e of the library's own u_L and w_{L-1} (e = u_L - w_{L-1} on each cell's closure,
    M_T from a one-cell oracle hierarchy), every cell agrees to 1e-12 relative: the pair arithmetic
    keeps about 2^-44 per node, far inside the 1e-10 of the oracle comparisons."""
    co, ce, L, k, h, mesh, maps = setup_case(P, name)
    f, g = fg(co.shape[1])
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    u = mesh.solve(nu=2, pre=2, post=1, n_extra=1)
    w = mesh.get_vector(1, L - 1)
    est = mesh.estimate(1)
    nc, dim = len(ce), co.shape[1]
    Nt = len(x) // nc
    worst = 0.0
    for T in range(nc):
        lev = O.Hierarchy(co[ce[T]], np.arange(dim + 1)[None, :], L).levels[L]
        sl = slice(T * Nt, (T + 1) * Nt)
        dist, idx = cKDTree(x[sl]).query(lev.x)
        assert dist.max() < 1e-9
        e = (u[sl] - w[sl])[idx]
        ref = float(e @ (lev.M @ e))
        worst = max(worst, abs(est["eta_T"][T] ** 2 - ref) / ref)
    assert worst <= 1e-12, worst


@pytest.mark.parametrize("name", ["lshape", "cube"])
def test_level_coords_device_path_matches_host_path(P, name):
    """hhg_level_coords into device memory (one kernel) gives the host path's coordinates bit for
    bit, on every level of a general mesh; both match the oracle's node coordinates."""
    import torch
    co, ce = perturbed(name)
    L = 4 if name == "lshape" else 3
    mesh = P.Mesh(co, ce, L)
    h = O.Hierarchy(co, ce, L)
    for lev in range(L + 1):
        xh = mesh.level_coords(lev)
        xd = torch.empty((mesh.n_nodes(lev), co.shape[1]), dtype=torch.float64, device="cuda")
        mesh.level_coords(lev, out=xd)
        assert np.array_equal(xd.cpu().numpy(), xh)
        dist, _ = cKDTree(h.levels[lev].x).query(xh)
        assert dist.max() < 1e-12
    mesh.close()


DEGENERATE = {
    # two macro triangles of the unit square: all four macro vertices on the Dirichlet boundary
    "two_triangles": lambda: (*W.square_mesh(1), 5),
    # one general macro tet: every vertex, edge and face on the Dirichlet boundary
    "one_tet": lambda: (np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.0], [0.3, 0.25, 0.8]]),
                        np.array([[0, 1, 2, 3]]), 4),
}


@pytest.mark.parametrize("name", list(DEGENERATE))
def test_coarse_grid_without_unknowns(P, name):
    """Degenerate coarse grid: level 0 has no unknown, so the direct coarse solve is empty and every
    V-cycle bottoms out on level 1.  FMG u_L, the stored w_l, the estimator for j = 1, 2 and the
    marking match the oracle, and the mixed-precision refinement (binary32 storage) converges to the
    exact discrete solution."""
    co, ce, L = DEGENERATE[name]()
    h = O.Hierarchy(co, ce, L)
    assert not h.levels[0].free.any() and h.levels[L].free.any()
    mesh = P.Mesh(co, ce, L)
    maps = []
    for l in range(L + 1):
        dist, idx = cKDTree(h.levels[l].x).query(mesh.level_coords(l))
        assert dist.max() < 1e-9
        maps.append(idx)
    f, g = fg(h.dim)
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    u = mesh.solve(nu=2, pre=2, post=1)
    prob = O.Problem(h, f, g)
    uo, ws, _ = O.fmg(prob, 2, 2, 1)
    close(u, uo[maps[L]])
    for l in range(L):
        close(mesh.get_vector(1, l), ws[l][maps[l + 1]])
    for j in (1, 2):
        eg = mesh.estimate(j)
        eo = O.estimate(h, uo, ws, j)
        close_estimates(eg, eo, h, uo)
        assert np.array_equal(P.mark(eg["eta_T"], 0.5), O.mark_top_fraction(eo["eta_T"], 0.5))
    um = mesh.solve(nu=2, pre=2, post=1, precision=1, storage=0, ir_steps=12, ir_vcycles=2)
    ex = O.exact_solve(prob)
    assert np.abs(um - ex[maps[L]]).max() <= 1e-10 * np.abs(ex).max()
    mesh.close()
