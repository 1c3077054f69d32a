"""Seeded synthetic inputs for the HHG full-multigrid workloads.

This module holds inputs only: coarse (macro) meshes, manufactured source and
boundary functions, and per-macro diffusion coefficients drawn from a
counter-based generator.  It contains none of the solver's arithmetic, so both
the CPU oracle and the CUDA path may take their inputs from here.

Workloads (sizes follow the paper's experiments, Sec. 5.1-5.4):

* ``square``   unit square, 2x2 squares each split by a "/" diagonal into two
               triangles (8 macro triangles); u = sin(pi x) sin(pi y).
* ``lshape``   L-shaped domain (-1,1)^2 minus [0,1]x[-1,0] (Sec. 5.2, Example
               5.2), 3 unit squares x 4 half-squares x 2 triangles = 24 macro
               triangles; Dirichlet data r^(2/3) sin(2 phi/3), f = 0.
* ``cube``     unit cube, m^3 cubes each split into 6 Kuhn tetrahedra along the
               main diagonal (m=4: 384 macro tets, m=8: 3072).
* ``fichera``  unit cube minus the octant [0,1/2]^3, 56 cubes of side 1/4 x 6
               Kuhn tetrahedra = 336 macro tets.
* ``waves``    the oscillating manufactured solution of Example 5.1.

The coefficient draws use SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): top 53 bits of each output give a
double in [0,1), taken in cell order.
"""

from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "square_mesh", "lshape_mesh", "cube_mesh", "fichera_mesh",
    "splitmix64_uniform", "coeff_loguniform", "coeff_uniform",
    "sin_product_u", "sin_product_f", "lshape_g", "waves_u", "waves_f",
    "WORKLOADS", "workload",
]

_MASK64 = (1 << 64) - 1


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0,1) from SplitMix64 started at `seed` (top 53 bits / 2^53)."""
    out = np.empty(n, dtype=np.float64)
    state = seed & _MASK64
    for i in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        z = z ^ (z >> 31)
        out[i] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def coeff_loguniform(n_cells: int, seed: int = 0, lo_exp: float = -2.0, hi_exp: float = 2.0) -> np.ndarray:
    """k_T = 10^U(lo_exp, hi_exp) per macro cell, in cell order."""
    u = splitmix64_uniform(seed, n_cells)
    return np.power(10.0, lo_exp + (hi_exp - lo_exp) * u)


def coeff_uniform(n_cells: int, seed: int = 1, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """k_T = U(lo, hi) per macro cell, in cell order."""
    return lo + (hi - lo) * splitmix64_uniform(seed, n_cells)


def _grid_mesh_2d(squares):
    """Triangulate unit-size squares given by their lower-left corners (in units of h).

    Each square (a=(x,y), b=(x+1,y), c=(x+1,y+1), d=(x,y+1)) is split along the
    "/" diagonal a-c into triangles (a,b,c) and (a,c,d).
    """
    index = {}
    coords = []

    def vid(p):
        if p not in index:
            index[p] = len(coords)
            coords.append(p)
        return index[p]

    cells = []
    for (x, y) in squares:
        a, b, c, d = vid((x, y)), vid((x + 1, y)), vid((x + 1, y + 1)), vid((x, y + 1))
        cells.append((a, b, c))
        cells.append((a, c, d))
    return np.array(coords, dtype=np.float64), np.array(cells, dtype=np.int32)


def square_mesh(m: int = 2):
    """Unit square, m x m squares, 2 m^2 macro triangles."""
    co, ce = _grid_mesh_2d([(x, y) for y in range(m) for x in range(m)])
    return co / m, ce


def lshape_mesh():
    """(-1,1)^2 minus [0,1]x[-1,0]: 12 squares of side 1/2, 24 macro triangles."""
    sq = [(x, y) for y in range(-2, 2) for x in range(-2, 2) if not (x >= 0 and y < 0)]
    co, ce = _grid_mesh_2d(sq)
    return co / 2.0, ce


_KUHN_PERMS = list(itertools.permutations(range(3)))


def _kuhn_cubes(cubes):
    """Split unit cubes (lower corners, in units of h) into 6 Kuhn tets each.

    Tet for permutation s: (c, c+e_s0, c+e_s0+e_s1, c+(1,1,1)).
    """
    index = {}
    coords = []

    def vid(p):
        if p not in index:
            index[p] = len(coords)
            coords.append(p)
        return index[p]

    cells = []
    for c in cubes:
        for s in _KUHN_PERMS:
            p = list(c)
            verts = [vid(tuple(p))]
            for a in s:
                p = p[:]
                p[a] += 1
                verts.append(vid(tuple(p)))
            cells.append(verts)
    return np.array(coords, dtype=np.float64), np.array(cells, dtype=np.int32)


def cube_mesh(m: int = 4):
    """Unit cube, m^3 cubes x 6 Kuhn tets = 6 m^3 macro tets."""
    co, ce = _kuhn_cubes([(x, y, z) for z in range(m) for y in range(m) for x in range(m)])
    return co / m, ce


def fichera_mesh():
    """Unit cube minus [0,1/2]^3: 56 cubes of side 1/4 x 6 tets = 336 macro tets."""
    cubes = [(x, y, z) for z in range(4) for y in range(4) for x in range(4)
             if not (x < 2 and y < 2 and z < 2)]
    co, ce = _kuhn_cubes(cubes)
    return co / 4.0, ce


def perturbed_mesh(name: str, seed: int = 4, amp: float = 0.12, m: int = 2):
    """General (non-lattice) macro meshes: the L-shape ("lshape") or the m^3 Kuhn cube ("cube") with
    every vertex off the boundary (and, for the L-shape, off the axes through the re-entrant corner)
    moved by amp * h * U(-1, 1) per coordinate (numpy default_rng(seed)), h = 1/2 for the L-shape and
    1/m for the cube.  Triangles / tets then have full 7- / 15-point stencils."""
    co, ce = lshape_mesh() if name == "lshape" else cube_mesh(m)
    co = co.copy()
    rng = np.random.default_rng(seed)
    h = 0.5 if name == "lshape" else 1.0 / m
    inner = np.all(np.abs(co) < 1 - 1e-9, axis=1) if name == "lshape" else \
        np.all((co > 1e-9) & (co < 1 - 1e-9), axis=1)
    if name == "lshape":
        inner &= ~((np.abs(co[:, 0]) < 1e-9) | (np.abs(co[:, 1]) < 1e-9))
    co[inner] += amp * h * rng.uniform(-1, 1, size=(inner.sum(), co.shape[1]))
    return co, ce


# ---- manufactured functions (evaluated at points x of shape (N, d)) ----

def sin_product_u(x: np.ndarray) -> np.ndarray:
    return np.prod(np.sin(np.pi * x), axis=1)


def sin_product_f(x: np.ndarray) -> np.ndarray:
    d = x.shape[1]
    return d * np.pi ** 2 * np.prod(np.sin(np.pi * x), axis=1)


def lshape_g(x):
    """r^(2/3) sin(2 phi / 3) with phi in [0, 2 pi) measured from the +x axis (numpy or torch)."""
    if isinstance(x, np.ndarray):
        hypot, atan2, where, sin = np.hypot, np.arctan2, np.where, np.sin
    else:
        import torch
        hypot, atan2, where, sin = torch.hypot, torch.atan2, torch.where, torch.sin
    r = hypot(x[:, 0], x[:, 1])
    phi = atan2(x[:, 1], x[:, 0])
    phi = where(phi < 0.0, phi + 2.0 * np.pi, phi)
    return r ** (2.0 / 3.0) * sin(2.0 * phi / 3.0)


def _fns(x):
    """(exp, cos, sin) for a numpy array or a torch tensor (device inputs of large workloads)."""
    if isinstance(x, np.ndarray):
        return np.exp, np.cos, np.sin
    import torch
    return torch.exp, torch.cos, torch.sin


def _waves_w(t, omega, alpha):
    exp, cos, _ = _fns(t)
    return 1.0 - cos(exp(alpha * (t - 1.0)) * omega * t)


def _waves_w2(t, omega, alpha):
    # second derivative of 1 - cos(s(t)), s = exp(alpha (t-1)) omega t
    exp, cos, sin = _fns(t)
    e = exp(alpha * (t - 1.0))
    s = e * omega * t
    ds = omega * e * (1.0 + alpha * t)
    d2s = omega * e * (2.0 * alpha + alpha * alpha * t)
    return cos(s) * ds * ds + sin(s) * d2s


def waves_u(x, omega=16 * np.pi, alpha=10.0):
    """u = prod_i w(x_i), w(t) = 1 - cos(exp(alpha (t - 1)) omega t) (Example 5.1, extended to d
    dims as in the scaling study of Sec. 5.4); x: (N, d) numpy array or torch tensor."""
    w = _waves_w(x, omega, alpha)
    u = w[:, 0]
    for i in range(1, x.shape[1]):
        u = u * w[:, i]
    return u


def waves_f(x, omega=16 * np.pi, alpha=10.0):
    """-Laplace(u) for u = prod_i w(x_i) (Example 5.1, extended to d dims)."""
    w = _waves_w(x, omega, alpha)
    w2 = _waves_w2(x, omega, alpha)
    d = x.shape[1]
    f = 0.0 * w[:, 0]
    for i in range(d):
        t = w2[:, i]
        for j in range(d):
            if j != i:
                t = t * w[:, j]
        f = f - t
    return f


def _zero(x):
    if isinstance(x, np.ndarray):
        return np.zeros(x.shape[0])
    return x.new_zeros(x.shape[0])


def _one(x):
    if isinstance(x, np.ndarray):
        return np.ones(x.shape[0])
    return x.new_ones(x.shape[0])


# name -> (mesh builder, finest level L, f, g, coefficient builder or None, exact u or None)
WORKLOADS = {
    # 2D Poisson, 8 macro triangles, L=4 (small parity case)
    "square_l4": dict(mesh=lambda: square_mesh(2), L=4, f=sin_product_f, g=_zero, k=None, u=sin_product_u),
    # L-shape, 24 macro triangles, L=7, four k-refinement steps marking the top 20 %
    "lshape_l7": dict(mesh=lshape_mesh, L=7, f=_zero, g=lshape_g, k=None, u=lshape_g),
    # unit cube, 384 Kuhn tets, L=6, sin-product solution
    "cube384_l6": dict(mesh=lambda: cube_mesh(4), L=6, f=sin_product_f, g=_zero, k=None, u=sin_product_u),
    # unit cube, 3072 Kuhn tets, L=7, f=1, k log-uniform in [1e-2,1e2] (SplitMix64 seed 0)
    "cube3072_l7": dict(mesh=lambda: cube_mesh(8), L=7, f=_one, g=_zero,
                        k=lambda n: coeff_loguniform(n, seed=0), u=None),
    # unit cube, 3^3 cubes x 6 Kuhn tets = 162 tets, L=8, waves solution (omega = 16 pi, alpha = 10):
    # the one-node size of the scaling program of Sec. 5.4 (Alg. 5, refinement of 12.5 %)
    "waves3d_l8": dict(mesh=lambda: cube_mesh(3), L=8, f=waves_f, g=waves_u, k=None, u=waves_u),
    # Fichera corner, 336 tets, L=6, f=1, k uniform in [0.5,2] (SplitMix64 seed 1)
    "fichera336_l6": dict(mesh=fichera_mesh, L=6, f=_one, g=_zero,
                          k=lambda n: coeff_uniform(n, seed=1), u=None),
}


def workload(name: str, L: int | None = None):
    """Return (coords, cells, L, f, g, k_per_cell or None, u_exact or None)."""
    w = WORKLOADS[name]
    coords, cells = w["mesh"]()
    k = w["k"](len(cells)) if w["k"] is not None else None
    return coords, cells, (w["L"] if L is None else L), w["f"], w["g"], k, w["u"]
