"""torch.autograd wrapper of the adjoint solve (paper_2508_06049_gb300.autograd): the gradients that
backward() delivers equal the library's adjoint gradients, and J matches the oracle's exact value."""

import numpy as np
import pytest

import workloads as W
from oracle import hhg_oracle as O

pytestmark = pytest.mark.gpu


def test_l2_functional_backward_matches_adjoint():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06049_gb300 as P
    from paper_2508_06049_gb300.autograd import l2_functional
    co, ce = W.fichera_mesh()
    L = 3
    k0 = W.coeff_uniform(len(ce), seed=1)
    mesh = P.Mesh(co, ce, L)
    x = mesh.level_coords(L)
    dev = torch.device("cuda:0")
    f = torch.tensor(np.sin(3 * x[:, 0]) + x[:, 2], dtype=torch.float64, device=dev, requires_grad=True)
    k = torch.tensor(k0, dtype=torch.float64, requires_grad=True)
    in_S = np.all(co[ce].mean(axis=1) > 0.5, axis=1)
    prm = P.solve_params(n_extra=40)
    J = l2_functional(f, k, mesh, in_S, params=prm)
    J.backward()
    # the same through the plain binding
    mesh.set_coefficient(k0)
    mesh.set_data(f.detach().cpu().numpy(), np.zeros(len(x)))
    mesh.solve(prm)
    Jr, gf, gk = mesh.adjoint_l2(in_S, params=prm)
    assert abs(J.item() - Jr) <= 1e-12 * abs(Jr)
    np.testing.assert_allclose(f.grad.cpu().numpy(), gf, rtol=0, atol=1e-12 * np.abs(gf).max())
    np.testing.assert_allclose(k.grad.numpy(), gk, rtol=0, atol=1e-12 * np.abs(gk).max())
    # and J against the oracle's exact discrete solution
    h = O.Hierarchy(co, ce, L, k=k0)
    fo = lambda y: np.sin(3 * y[:, 0]) + y[:, 2]
    uo = O.exact_solve(O.Problem(h, fo, lambda y: np.zeros(len(y))))
    Jo, _, _, _ = O.adjoint_gradients(h, uo, in_S)
    assert abs(J.item() - Jo) <= 1e-9 * abs(Jo)
    mesh.close()


def test_source_gradient_is_the_derivative_by_each_copy():
    """dJ/df_L is the derivative by each entry of the level-L layout: for one copy of an interface
    node it equals the central difference of J in that entry alone (J is quadratic in f, so the
    difference is exact up to the solve's algebraic error), the copies of a node differ, and
    backpropagating through f_L = f_nodes[idx] gives the oracle's derivative by the nodal value.
    Without gradients the forward evaluates J from the solution alone, to the same value."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from scipy.spatial import cKDTree

    import paper_2508_06049_gb300 as P
    from paper_2508_06049_gb300.autograd import l2_functional
    co, ce = W.fichera_mesh()
    L = 3
    k0 = W.coeff_uniform(len(ce), seed=1)
    mesh = P.Mesh(co, ce, L)
    x = mesh.level_coords(L)
    h = O.Hierarchy(co, ce, L, k=k0)
    _, idx = cKDTree(h.levels[L].x).query(x)
    dev = torch.device("cuda:0")
    fo = lambda y: np.sin(3 * y[:, 0]) + y[:, 2]
    in_S = np.all(co[ce].mean(axis=1) > 0.5, axis=1)
    prm = P.solve_params(n_extra=60)
    k = torch.tensor(k0, dtype=torch.float64)
    f_nodes = torch.tensor(fo(h.levels[L].x), dtype=torch.float64, device=dev, requires_grad=True)
    J = l2_functional(f_nodes[torch.as_tensor(idx, device=dev)], k, mesh, in_S, params=prm)
    J.backward()
    Jo, gfo, _, _ = O.adjoint_gradients(h, O.exact_solve(O.Problem(h, fo, lambda y: np.zeros(len(y)))), in_S)
    assert abs(J.item() - Jo) <= 1e-9 * abs(Jo)
    assert np.abs(f_nodes.grad.cpu().numpy() - gfo).max() <= 1e-9 * np.abs(gfo).max()
    # one copy of a free interface node shared by several cells
    f = torch.tensor(fo(x), dtype=torch.float64, device=dev, requires_grad=True)
    Jf = l2_functional(f, k, mesh, in_S, params=prm)
    Jf.backward()
    g = f.grad.cpu().numpy()
    cnt = np.bincount(idx)
    free = h.levels[L].free[idx]
    c = int(np.nonzero((cnt[idx] > 2) & free & (np.abs(g) > 1e-3 * np.abs(g).max()))[0][0])
    others = np.nonzero(idx == idx[c])[0]
    assert len(others) > 2 and np.ptp(g[others]) > 1e-6 * abs(g[c])      # the copies' shares differ
    assert abs(g[others].sum() - gfo[idx[c]]) <= 1e-9 * np.abs(gfo).max()
    d = 1e-2 * max(1.0, abs(float(f[c])))
    with torch.no_grad():
        fp = f.detach().clone()
        fp[c] += d
        Jp = l2_functional(fp, k, mesh, in_S, params=prm).item()
        fm = f.detach().clone()
        fm[c] -= d
        Jm = l2_functional(fm, k, mesh, in_S, params=prm).item()
        J0 = l2_functional(f.detach(), k, mesh, in_S, params=prm).item()
    assert abs(J0 - Jf.item()) <= 1e-12 * abs(Jf.item())
    fd = (Jp - Jm) / (2 * d)
    assert abs(fd - g[c]) <= 1e-6 * np.abs(g).max(), (fd, g[c])
    mesh.close()
