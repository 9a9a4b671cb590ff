"""Measure the device peaks the solver's roofline uses besides the copy
bandwidth: FP64 / FP32 FMA throughput and L2-resident read bandwidth.

    python -m paper_2501_08293_b300.probe
"""
import os
import subprocess
import sys

from .build import ARCH, nvcc

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    src = os.path.join(HERE, "probe_src", "peaks.cu")
    exe = os.path.join(HERE, "probe_src", "peaks")
    subprocess.run([nvcc(), *ARCH, "-O3", "-o", exe, src], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    sys.stderr.write(r.stderr)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
