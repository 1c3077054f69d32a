"""Build libhhg.so (the C-ABI library) in-tree for sm_103a with nvcc.

Translation units are compiled in parallel; the result goes to paper_2508_06049_gb300/lib/.  Host
code is compiled with -ffp-contract=off: without it GCC fuses multiply-adds on Arm but not on x86,
and host results (stencils, coordinates, refined meshes) would differ between the two in the last
bit.
Usage: python -m paper_2508_06049_gb300.build [--debug]
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
BUILD = os.path.join(HERE, "_build")
LIBNAME = "libhhg.so"

CUDA_SOURCES = ["setup.cu", "kernels.cu", "kernels_mixed.cu", "kernels_noalloc.cu", "capi.cu"]
CXX_SOURCES = ["rg2d.cpp", "rg3d.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r


def build(debug: bool = False, verbose: bool = False, check: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    opt = ["-O0", "-g"] if debug else ["-O3"]
    common = opt + ["-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-pthread,-ffp-contract=off", "-I", CSRC]
    if check or os.environ.get("HHG_CHECK"):
        common += ["-DHHG_CHECK=1"]
    jobs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append([nvcc] + ARCH + common + ["-c", os.path.join(CSRC, src), "-o", obj])
    cxx = shutil.which("g++") or "g++"
    for src in CXX_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append([cxx] + opt + ["-std=c++17", "-fPIC", "-ffp-contract=off", "-c", os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        for r in ex.map(_run, jobs):
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr)
    objs = [os.path.join(BUILD, s + ".o") for s in CUDA_SOURCES + CXX_SOURCES]
    out = os.path.join(LIBDIR, LIBNAME)
    tmp = out + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(debug="--debug" in sys.argv, verbose=True, check="--check" in sys.argv))
