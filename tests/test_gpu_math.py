"""The step kernel's own arithmetic helpers against CUDA's IEEE operations:
Newton-refined reciprocal and reciprocal square root (FP64) within a few
ulp, and the integer-unit double<->float conversions (exact float->double;
double->float within one float ulp of round-to-nearest)."""
import ctypes

import numpy as np
import pytest

from paper_1712_07070_b300 import amr_hydro as A

pytestmark = pytest.mark.gpu


def test_math_helpers_against_ieee():
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 20000), rng.uniform(0.5, 2.0, 20000),
                        [1.0, 2.0, 0.1, 3.0, 1e-37, 1e37, 7.0 / 3.0]])
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(8 * len(x), dtype=torch.float64, device="cuda")
    fn = A.lib().amrh_selftest_math
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert fn(xd.data_ptr(), len(x), out.data_ptr()) == 0
    o = out.cpu().numpy().reshape(-1, 8)
    ulp = np.spacing(np.abs(o[:, 1]))
    assert (np.abs(o[:, 0] - o[:, 1]) <= 2 * ulp).all()
    ulp = np.spacing(np.abs(o[:, 3]))
    assert (np.abs(o[:, 2] - o[:, 3]) <= 4 * ulp).all()
    inrange = (x > 1.2e-38) & (x < 3e38)
    fulp = np.spacing(np.abs(o[:, 5]).astype(np.float32)).astype(np.float64)
    assert (np.abs(o[inrange, 4] - o[inrange, 5]) <= fulp[inrange]).all()
    assert np.array_equal(o[:, 6], o[:, 7])
