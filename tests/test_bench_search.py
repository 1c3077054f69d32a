"""The benchmark's equal-error search (host logic, no GPU): `least_passing` finds the least passing
count of a monotone criterion, and `equal_error_search` applies the two-digit rule to each arm and
keeps the faster of the mixed arm's two passing (steps, V-cycles) pairs.  A fake mesh stands in for
the library: its solves return the exact solution plus an error that shrinks with the work done, and
its mixed solves take time in proportion to their V-cycles and refinement residuals."""

import math
import time
from types import SimpleNamespace

import numpy as np
import pytest

import bench

torch = pytest.importorskip("torch")


def test_least_passing_finds_the_threshold():
    for hi in (1, 7, 24, 64, 160):
        for t in range(0, hi + 3):
            calls = []

            def ok(n):
                calls.append(n)
                return n >= t

            got = bench.least_passing(ok, hi)
            assert got == (t if t <= hi else None), (hi, t, got)
            assert len(calls) <= 2 * math.ceil(math.log2(hi + 1)) + 2


class FakeMesh:
    """err(binary64, n extra) = e0 (1 + 0.5^n); err(mixed, s steps of v V-cycles) = e0 (1 + 0.45^(s v));
    a mixed solve sleeps (v + 3) ms per step (a refinement residual costs three V-cycles here)."""

    def __init__(self, n, e0=1e-3):
        self.n_cells, self.n, self.e0 = 1, n, e0
        self.ue = torch.linspace(0.0, 1.0, n, dtype=torch.float64)

    def solve(self, p, out):
        if p.precision == 0:
            rel = 0.5 ** p.n_extra
        else:
            rel = 0.45 ** (p.ir_steps * p.ir_vcycles)
            time.sleep(1e-3 * p.ir_steps * (p.ir_vcycles + 3))
        out.copy_(self.ue)
        out[0] += self.e0 * (1.0 + rel)
        return out

    def cell_mass_norms_noalloc(self, a, b, cells):
        cells[0] = float(((a - b) ** 2).sum())

    def synchronize(self):
        pass

    def estimate(self, j, want_local=True):
        return {"eta_j": 2.0 * self.e0}


def _params(**kw):
    return SimpleNamespace(**kw)


def test_equal_error_search_with_an_exact_solution():
    mesh = FakeMesh(16)
    P = SimpleNamespace(solve_params=_params)
    su = SimpleNamespace(mesh=mesh, s=None, fd=torch.zeros(16, dtype=torch.float64), ued=mesh.ue.clone())
    res = bench.equal_error_search(su, P, storage=0)
    # binary64: |e0 (1 + 0.5^n) - e0 (1 + 0.5^24)| <= 1 % of e_ref first for n = 7
    assert res["fp64"]["n_extra"] == 7
    # mixed: 0.45^(s v) <= 1 % first for s v = 6: 6 x 1 (24 ms) or 3 x 2 (15 ms); the faster is kept
    assert (res["mixed"]["ir_steps"], res["mixed"]["ir_vcycles"]) == (3, 2)
    assert res["mixed"]["solve_seconds"]["3x2"] < res["mixed"]["solve_seconds"]["6x1"]
    for key, e in res["mixed"]["tried_steps_x_vcycles"].items():
        s, v = map(int, key.split("x"))
        assert math.isclose(e, mesh.e0 * (1 + 0.45 ** (s * v)), rel_tol=1e-12)


def test_equal_error_search_without_an_exact_solution():
    """Algebraic criterion: ||u_L - u_ref|| <= 1 % of eta_1 (here 2 e0) with u_ref the binary64 solve
    with REF_EXTRA_ALG extra V-cycles: |0.5^n - 0.5^160| e0 <= 0.02 e0 first at n = 6."""
    mesh = FakeMesh(16)
    P = SimpleNamespace(solve_params=_params)
    su = SimpleNamespace(mesh=mesh, s=None, fd=torch.zeros(16, dtype=torch.float64), ued=None)
    res = bench.equal_error_search(su, P, storage=1)
    assert res["fp64"]["n_extra"] == 6
    assert res["reference_error"] is None
    # mixed: |0.45^(s v) - 0.5^160| <= 0.02 first at s v = 5 (0.45^5 = 0.0185): 5 x 1 or 3 x 2
    # (3 x 2 = 6 V-cycles, 15 ms; 5 x 1 = 20 ms): the faster is 3 x 2
    assert (res["mixed"]["ir_steps"], res["mixed"]["ir_vcycles"]) == (3, 2)
    assert res["mixed"]["storage"] == 1
