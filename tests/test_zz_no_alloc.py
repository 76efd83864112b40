"""The allocation-free uniform step, for callers that cannot call cudaMalloc
(their device memory is reserved up front by their own pool allocator, or a
latency-critical loop cannot take the device-wide synchronisation an
allocation may cause).  Its scratch is a static device array, so its output
must equal the regular context-based entry point's on consecutive calls.

This file is collected last on purpose: the GPU test must pass both alone in
a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics

G53 = 5.0 / 3.0


def test_noalloc_rejects_sizes_beyond_static_scratch():
    # validation happens before any device work: 512^3 is 32768 groups > 4096
    st = A.lib().amr_hydro_step_uniform_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(32), 512, 512, 512,
                                                1.0 / 512, 1e-4, G53, 0.5, A.AMR_FP64, None, None, None)
    assert st == A.AMR_E_INVAL
    st = A.lib().amr_hydro_step_uniform_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(32), 40, 32, 32,
                                                1.0 / 40, 1e-4, G53, 0.5, A.AMR_FP64, None, None, None)
    assert st == A.AMR_E_INVAL


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [A.AMR_FP64, A.AMR_FP32_ACC64])
def test_noalloc_matches_context_entry_point_two_calls(prec):
    import torch
    from paper_1712_07070_b300.uniform import UniformGrid

    nx, ny, nz = 64, 32, 48
    U0 = ics.sod_noise(nx, seed=3, ny=ny, nz=nz)
    g = UniformGrid((nx, ny, nz), prec=prec)
    g.upload(U0)
    # caller-owned buffers for the allocation-free path, same patch layout
    a = g.state().clone()
    b = torch.empty_like(a)
    dt_next = torch.empty(1, dtype=torch.float64, device="cuda")
    nbad = torch.zeros(1, dtype=torch.int64, device="cuda")
    for call in range(2):
        dt = g.min_dt()
        g.step(dt)
        A.amr_hydro_step_uniform_noalloc(a, b, nx, ny, nz, g.dh, dt, G53, 0.5, prec, dt_next, nbad)
        torch.cuda.synchronize()
        ref = g.state()
        # the same kernel on the same data: every cell agrees bit for bit
        # (tighter than the 1e-12 / 1e-5 oracle tolerances of the other tests)
        assert torch.equal(b, ref), (call, (b - ref).abs().max().item())
        assert int(nbad.item()) == 0
        assert abs(dt_next.item() - g.min_dt()) <= 1e-14 * g.min_dt()
        a, b = b, a
    g.close()
