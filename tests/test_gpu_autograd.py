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
