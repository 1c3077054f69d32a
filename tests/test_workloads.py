"""Input generators: the manufactured sources are the negative Laplacians of their solutions, the
device (torch) and host (numpy) evaluations agree, and the meshes have the stated sizes."""

import numpy as np
import pytest

import workloads as W


def _neg_laplacian_fd(u, x, h):
    """Second-order central differences of -Laplace(u) at the points x."""
    d = x.shape[1]
    lap = np.zeros(len(x))
    for i in range(d):
        e = np.zeros(d)
        e[i] = h
        lap += (u(x + e) - 2 * u(x) + u(x - e)) / h ** 2
    return -lap


@pytest.mark.parametrize("d", [2, 3])
def test_waves_source_is_negative_laplacian(d):
    rng = np.random.default_rng(3)
    x = rng.uniform(0.05, 0.95, size=(200, d))
    f = W.waves_f(x)
    fd = _neg_laplacian_fd(W.waves_u, x, 1e-4)
    # the solution oscillates with frequency up to omega e^0 (1 + alpha) ~ 550: the difference
    # quotient's error is ~ h^2 u''''/12 relative to f's scale
    assert np.abs(f - fd).max() <= 1e-4 * np.abs(f).max()


def test_waves_boundary_values_vanish():
    # w(0) = 0 and w(1) = 1 - cos(16 pi) = 0: the solution is zero on the cube's boundary
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, size=(50, 3))
    for dd in range(3):
        for v in (0.0, 1.0):
            y = x.copy()
            y[:, dd] = v
            assert np.abs(W.waves_u(y)).max() < 1e-12


def test_sin_product_source_is_negative_laplacian():
    rng = np.random.default_rng(5)
    x = rng.uniform(0.05, 0.95, size=(100, 3))
    assert np.abs(W.sin_product_f(x) - _neg_laplacian_fd(W.sin_product_u, x, 1e-4)).max() < 1e-5


def test_waves_torch_matches_numpy():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 1, size=(300, 3))
    xt = torch.from_numpy(x)
    assert np.allclose(W.waves_u(xt).numpy(), W.waves_u(x), rtol=1e-13, atol=1e-13)
    assert np.allclose(W.waves_f(xt).numpy(), W.waves_f(x), rtol=1e-13, atol=1e-9)


def test_waves3d_mesh_is_the_162_tet_cube():
    co, ce, L, f, g, k, u = W.workload("waves3d_l8")
    assert len(ce) == 162 and L == 8 and len(co) == 64
    X = co[ce]
    vol = np.abs(np.einsum("ij,ij->i", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0])) / 6
    assert abs(vol.sum() - 1.0) < 1e-14
