"""Independent periodic boxes of uneven sizes in one persistent launch per
step, captured in a CUDA graph, per-box device dt (Eq. CFL2): every box must
match the oracle's own run, graph replays must continue the same evolution,
and every launch shape the autotuner may pick must give bit-identical
results."""
import os

import numpy as np
import pytest

import oracle
from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics

pytestmark = pytest.mark.gpu
G14 = 1.4


def rel_l1(a, b):
    ref = np.abs(b[0]).sum()
    return np.array([np.abs(a[v] - b[v]).sum() / (np.abs(b[v]).sum() or ref) for v in range(5)])


def batch(sizes, prec, seed0=10):
    from paper_1712_07070_b300.boxes import BoxBatch
    B = BoxBatch(gamma=G14, prec=prec)
    U0 = [ics.kh_box(n, seed=seed0 + i, gamma=G14) for i, n in enumerate(sizes)]
    for U in U0:
        B.add_box(U)
    return B, U0


@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 1e-5)])
def test_boxes_match_oracle_and_graph_replay(prec, tol):
    sizes = [32, 48, 16, 64]
    B, U0 = batch(sizes, prec)
    d1 = B.advance(3).cpu().numpy()
    d2 = B.advance(3).cpu().numpy()  # replays the captured graph
    for i, n in enumerate(sizes):
        ref, dts = oracle.run_periodic(U0[i], 1.0 / n, G14, 0.5, 6)
        err = rel_l1(B.download(i), ref)
        assert (err <= tol).all(), (n, err)
        got = np.concatenate([d1[:, i], d2[:, i]])
        assert np.allclose(got, dts, rtol=(1e-14 if prec == A.AMR_FP64 else 1e-6), atol=0), (n, got, dts)
    B.close()


def test_autotuned_shapes_are_bitwise_identical():
    sizes = [32, 48, 16]
    outs = []
    for env in ("0", "1"):
        os.environ["AMR_HYDRO_AUTOTUNE"] = env
        try:
            B, _ = batch(sizes, A.AMR_FP32_ACC64)
            B.advance(4)
            outs.append(([B.download(i) for i in range(len(sizes))], B.tuning()))
            B.close()
        finally:
            os.environ.pop("AMR_HYDRO_AUTOTUNE", None)
    for a, b in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(a, b)
    assert outs[1][1]["grid"] > 0


def test_boxes_run_to_run_bitwise():
    sizes = [32, 16]
    res = []
    for _ in range(2):
        B, _ = batch(sizes, A.AMR_FP64)
        B.advance(3)
        res.append([B.download(i) for i in range(2)])
        B.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_full_size_batch_in_the_benchmark_launch():
    """The benchmark's batch (64 KH boxes of seeded sizes {32..192}^3, FP32
    mode, one persistent autotuned launch per step, CUDA graph): after two
    steps every box of edge <= 48 matches the oracle (1e-5), and every box
    conserves mass, momentum and energy to FP32 round-off of its fluxes."""
    import torch
    from paper_1712_07070_b300.boxes import BoxBatch
    sizes = ics.kh_batch_sizes(64, seed=4)
    B = BoxBatch(gamma=G14, prec=A.AMR_FP32_ACC64)
    U0 = [ics.kh_box(n, seed=100 + i, gamma=G14) for i, n in enumerate(sizes)]
    for U in U0:
        B.add_box(U)
    B.advance(2)
    torch.cuda.synchronize()
    checked = 0
    for i, n in enumerate(sizes):
        out = B.download(i)
        s0 = U0[i].reshape(5, -1).sum(1)
        s1 = out.reshape(5, -1).sum(1)
        l1 = np.abs(U0[i]).reshape(5, -1).sum(1)
        assert (np.abs(s1 - s0) <= 1e-6 * np.maximum(l1, l1[0])).all(), (n, s1 - s0)
        if n <= 48:
            ref, _ = oracle.run_periodic(U0[i], 1.0 / n, G14, 0.5, 2)
            err = rel_l1(out, ref)
            assert (err <= 1e-5).all(), (n, err)
            checked += 1
    assert checked > 0
    B.close()
