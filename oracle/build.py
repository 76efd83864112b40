"""Compile the C oracle into oracle/liboracle.so.

The oracle is test infrastructure: it is built here so that the tests, the
smoke check and the CPU-baseline leg of the benchmark can load it; the CUDA
product path never links or calls it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["hydro_oracle.c", "amr_oracle.c"]
LIB = os.path.join(HERE, "liboracle.so")
# -ffp-contract=off: no fused multiply-adds, so every operation rounds exactly
# as written; no -march=native: the library must also run on another host.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


FLOPLIB = os.path.join(HERE, "libflopcount.so")
ADLIB = os.path.join(HERE, "liboracle_ad.so")


def _stale(lib, srcs):
    if not os.path.exists(lib):
        return True
    m = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > m for s in srcs)


def build(force=False):
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    if force or _stale(LIB, srcs):
        subprocess.run(["gcc", *CFLAGS, "-o", LIB, *srcs, "-lm"], check=True)
    fsrc = [os.path.join(HERE, "flop_count.cpp"), os.path.join(HERE, "hydro_oracle.c")]
    if force or _stale(FLOPLIB, fsrc):
        # the counting build: no OpenMP (its pragmas are ignored), C++ for the
        # operator-overloaded counting type
        subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-Wno-unknown-pragmas",
                        "-o", FLOPLIB, fsrc[0]], check=True)
    asrc = [os.path.join(HERE, "adjoint_oracle.cpp"), os.path.join(HERE, "hydro_oracle.c")]
    if force or _stale(ADLIB, asrc):
        # the taping / dual-number builds: no OpenMP (the tape is sequential)
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                        "-Wno-unknown-pragmas", "-o", ADLIB, asrc[0]], check=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
