"""Host-side checks of bench.py: the algorithmic flop count it reports is the
instrumented oracle's, and the multi-rank timing reduction (max over ranks)
works on world_size-2 gloo ranks."""
import os
import socket
import subprocess
import sys

import pytest

import oracle
from paper_1712_07070_b300 import ics

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_alg_flops_constant_matches_instrumented_oracle():
    c = oracle.count_flops(ics.turbulence(16, seed=1), 5.0 / 3.0)
    per_cell = sum(c["step"][k] for k in ("add", "mul", "div", "sqrt")) + \
        sum(c["speed"][k] for k in ("add", "mul", "div", "sqrt"))
    assert abs(per_cell - bench.ALG_FLOPS_PER_CELL) <= 0.01 * bench.ALG_FLOPS_PER_CELL, per_cell


def test_fp64_peak_derivation():
    assert abs(bench.FP64_PEAK_TFLOPS - 1.2029) < 1e-3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import bench
rank, world = bench.dist_init("gloo")
t = 1.0 + rank
bench.barrier()
m = bench.max_over_ranks(t)
assert m == 1.0 + (world - 1), m
print("ok", rank, m)
"""


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        assert out.startswith("ok")
