"""The allocation-free per-cell mass-norm entry point (hhg_cell_mass_norms_noalloc).

Some callers cannot allocate device memory when they need the local indicators (a caller recording
its own CUDA stream capture, or one running under a fixed device-memory budget); this entry point
keeps its scratch in a file-scope device array instead.  Its output must equal the squared local
indicators eta_T^2 of hhg_estimate (the existing entry point) within the parity tolerance, on two
calls in a row (the shared scratch keeps the previous call's contents).  This file is collected last
so that a failure here does not hide the results of the other GPU tests.
"""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.mark.parametrize("name,L", [("lshape_l7", 5), ("cube384_l6", 4), ("fichera336_l6", 3)])
def test_noalloc_mass_norms_match_estimator(name, L):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06049_gb300 as P
    co, ce, _, f, g, k, _ = W.workload(name, L)
    s = torch.cuda.Stream()
    mesh = P.Mesh(co, ce, L, stream=s)
    if k is not None:
        mesh.set_coefficient(k)
    x = mesh.level_coords(L)
    mesh.set_data(np.ascontiguousarray(f(x)), np.ascontiguousarray(g(x)))
    n_L = mesh.n_nodes(L)
    with torch.cuda.stream(s):
        u = torch.empty(n_L, dtype=torch.float64, device="cuda")
        w = torch.empty(n_L, dtype=torch.float64, device="cuda")
        out = torch.full((len(ce),), float("nan"), dtype=torch.float64, device="cuda")
    mesh.solve(out=u)
    mesh.get_vector(1, L - 1, out=w)
    eta = mesh.estimate(1)["eta_T"]
    ref = eta ** 2
    for call in range(2):
        allocated = torch.cuda.memory_allocated()
        free_before = torch.cuda.mem_get_info()[0]
        mesh.cell_mass_norms_noalloc(u, w, out)
        s.synchronize()
        if call == 1:  # after the first call (kernel loading, symbol look-up) nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.cuda.memory_allocated() == allocated
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL * ref.max(), call
    # b = NULL: the norm of a itself, against the same entry point on the difference with zero
    zero = torch.zeros_like(u)
    mesh.cell_mass_norms_noalloc(u, None, out)
    s.synchronize()
    a_only = out.cpu().numpy().copy()
    mesh.cell_mass_norms_noalloc(u, zero, out)
    s.synchronize()
    assert np.abs(a_only - out.cpu().numpy()).max() <= TOL * a_only.max()
    # the binding rejects arguments the kernel would read out of bounds
    with torch.cuda.stream(s):
        bad = [u.float(), u[:-1], out[:-1].contiguous()]
    for a_, o_ in ((bad[0], out), (bad[1], out), (u, bad[2])):
        with pytest.raises(ValueError):
            mesh.cell_mass_norms_noalloc(a_, None, o_)
    with pytest.raises(ValueError):
        mesh.cell_mass_norms_noalloc(u.cpu(), None, out)
    mesh.close()
