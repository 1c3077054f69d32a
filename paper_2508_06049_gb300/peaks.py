"""Compile and run peak_probe.cu (binary64 / binary32 FMA throughput and copy bandwidth).

Usage: python -m paper_2508_06049_gb300.peaks  (needs a GPU; prints the probe's lines)
"""

import os
import subprocess
import sys

from .build import ARCH, PEAK_PROBE, _nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    exe = PEAK_PROBE
    if not os.path.exists(exe):  # build() compiles it; compile here when it has not run
        os.makedirs(os.path.dirname(exe), exist_ok=True)
        subprocess.run([_nvcc()] + ARCH + ["-O3", "-lineinfo", "-o", exe, os.path.join(HERE, "peak_probe.cu")],
                       check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
