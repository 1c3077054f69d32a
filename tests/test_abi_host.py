"""CPU tests of the C-ABI library: it loads, exports every symbol of include/hhg.h, and its host
logic (lattice index arithmetic, marking, 2D red-green refinement) matches the oracle bit for bit.
No GPU compute call is made here."""

import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import hhg_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_2508_06049_gb300 as pkg
    if not os.path.exists(pkg.hhg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return pkg


def test_library_exports_every_declared_symbol(P):
    header = open(os.path.join(ROOT, "include", "hhg.h")).read()
    names = set(re.findall(r"\b(hhg_[a-z0-9_]+)\s*\(", header))
    assert len(names) >= 18
    lib = P.lib()
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_every_exported_symbol_is_declared(P):
    """The reverse direction: the library's dynamic symbols named hhg_* are exactly the header's
    entry points (nothing leaks into the ABI undocumented)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", P.hhg.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.split() and line.split()[-1].startswith("hhg_")}
    header = open(os.path.join(ROOT, "include", "hhg.h")).read()
    declared = set(re.findall(r"\b(hhg_[a-z0-9_]+)\s*\(", header))
    assert exported == declared, (sorted(exported - declared), sorted(declared - exported))


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_index_arithmetic(P, dim):
    for n in (1, 2, 3, 4, 5, 8, 16, 32, 64):
        assert P.lattice_selfcheck(dim, n) == 0, n


def test_marking_matches_oracle(P):
    rng = np.random.default_rng(5)
    for trial in range(300):
        n = int(rng.integers(1, 60))
        eta = rng.random(n) * 10 ** rng.uniform(-6, 2)
        if trial % 4 == 0:
            eta[rng.integers(0, n, size=max(1, n // 3))] = eta[0]
        frac = float(rng.choice([0.1, 0.125, 0.2, 0.25, 1.0 / 3.0, 0.5, 1.0]))
        assert np.array_equal(P.mark(eta, frac), O.mark_top_fraction(eta, frac))


def test_marking_rejects_bad_input(P):
    with pytest.raises(P.HHGError):
        P.mark(np.array([1.0, np.nan]), 0.2)
    with pytest.raises(P.HHGError):
        P.mark(np.array([1.0, 2.0]), 0.0)


@pytest.mark.parametrize("mesh", ["lshape", "square"])
def test_red_green_matches_oracle(P, mesh):
    co, ce = W.lshape_mesh() if mesh == "lshape" else W.square_mesh(3)
    a = P.RG2D(co, ce)
    b = O.RG2D(co, ce)
    rng = np.random.default_rng(9)
    for step in range(6):
        c1, t1 = a.mesh()
        c2, t2 = b.mesh()
        assert np.array_equal(t1, t2) and np.array_equal(c1, c2), step
        eta = rng.random(len(t1))
        if step % 2:
            eta[: len(eta) // 2] = 0.5       # ties across many cells
        marked = a.mark_refine(eta, 0.2)
        assert np.array_equal(marked, O.mark_top_fraction(eta, 0.2))
        b.refine(marked)
    c1, t1 = a.mesh()
    c2, t2 = b.mesh()
    assert np.array_equal(t1, t2) and np.array_equal(c1, c2)


def test_gpu_entry_points_fail_cleanly_without_gpu(P):
    """Without a GPU, mesh creation must return an error status (no crash, no fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    co, ce = W.square_mesh(2)
    with pytest.raises(P.HHGError):
        P.Mesh(co, ce, 2)


def test_binding_argument_kinds_match_header():
    """Every entry point the Python binding declares has the header's parameter list: the same
    number of arguments and, position by position, the same kind (pointer or handle, int, double).
    A mismatch would pass garbage through ctypes, so this is checked without calling anything."""
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "hhg.h")).read(), flags=re.S)
    decls = {}
    for m in re.finditer(r"\b(?:hhg_status|int|const char\s*\*|void)\s+(hhg_\w+)\s*\(([^)]*)\)\s*;", hdr):
        kinds = []
        for a in m.group(2).split(","):
            a = a.strip()
            if not a or a == "void":
                continue
            if "*" in a or re.match(r"(const\s+)?hhg_(mesh|rg2d|rg3d)\b", a):
                kinds.append("ptr")
            elif re.match(r"(const\s+)?double\b", a):
                kinds.append("double")
            elif re.match(r"(const\s+)?(int|long long|unsigned)\b", a):
                kinds.append("int")
            else:
                kinds.append("?" + a)
        decls[m.group(1)] = kinds
    src = open(os.path.join(ROOT, "paper_2508_06049_gb300", "hhg.py")).read()
    start = src.index("sig = {")
    body = src[start:src.index("}", start)]
    kind_of = {"vp": "ptr", "u8": "ptr", "i": "int", "d": "double"}
    bound = dict()
    for m in re.finditer(r'"(hhg_\w+)":\s*\[([^\]]*)\]', body):
        toks = [t.strip() for t in m.group(2).split(",") if t.strip()]
        bound[m.group(1)] = ["ptr" if t.startswith("C.POINTER(") else kind_of.get(t, "?" + t) for t in toks]
    assert bound and set(bound) == set(decls), sorted(set(bound) ^ set(decls))
    for name, kinds in bound.items():
        assert kinds == decls[name], (name, kinds, decls[name])
