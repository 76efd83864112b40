"""Compile the C oracle into oracle/liboracle.so.

The oracle is test infrastructure: it is built here so that the tests, the
smoke check and the CPU-baseline leg of the benchmark can load it; the CUDA
product path never links or calls it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["hydro_oracle.c", "amr_oracle.c", "adjoint_oracle.c"]
LIB = os.path.join(HERE, "liboracle.so")
# -ffp-contract=off: no fused multiply-adds, so every operation rounds exactly
# as written; no -march=native: the library must also run on another host.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


def build(force=False):
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    if not force and os.path.exists(LIB):
        lib_m = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return LIB
    cmd = ["gcc", *CFLAGS, "-o", LIB, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
