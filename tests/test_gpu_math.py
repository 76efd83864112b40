"""The step kernel's own arithmetic helpers against CUDA's IEEE operations:
the refined reciprocal, reciprocal square root and square root (FP64) within
a few ulp (exact IEEE results at zeros, subnormals and negative inputs of the
square root), and the integer-unit double<->float conversions (exact
float->double; double->float within one float ulp of round-to-nearest)."""
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
    edge = np.array([0.0, -0.0, 5e-324, 1e-310, 2.2250738585072014e-308, 1.7976931348623157e308, -1.0])
    x = np.concatenate([x, edge])
    pos = x > 0
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(10 * len(x), dtype=torch.float64, device="cuda")
    fn = A.lib().amrh_selftest_math
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert fn(xd.data_ptr(), len(x), out.data_ptr()) == 0
    o = out.cpu().numpy().reshape(-1, 10)
    body = pos & (x >= 1e-300) & (x <= 1e300)  # reciprocals of the extremes leave the normal range
    ulp = np.spacing(np.abs(o[body, 1]))
    assert (np.abs(o[body, 0] - o[body, 1]) <= 2 * ulp).all()
    ulp = np.spacing(np.abs(o[body, 3]))
    assert (np.abs(o[body, 2] - o[body, 3]) <= 4 * ulp).all()
    # square root: a few ulp on positive normals, CUDA's own result elsewhere
    ulp = np.spacing(np.abs(o[pos, 9]))
    assert (np.abs(o[pos, 8] - o[pos, 9]) <= 4 * ulp).all()
    assert np.array_equal(o[~pos, 8], o[~pos, 9], equal_nan=True)
    assert np.array_equal(o[x == 0, 8], np.zeros((x == 0).sum())) and np.isnan(o[x == -1.0, 8]).all()
    inrange = (x > 1.2e-38) & (x < 3e38)
    fulp = np.spacing(np.abs(o[:, 5]).astype(np.float32)).astype(np.float64)
    assert (np.abs(o[inrange, 4] - o[inrange, 5]) <= fulp[inrange]).all()
    assert np.array_equal(o[inrange, 6], o[inrange, 7])


def test_integer_sign_tests_and_minmax():
    """The FP64 step's integer-unit sign tests and min/max agree with the
    FP64 comparisons on signed zeros, subnormals, infinities and random
    values of both signs."""
    import torch
    rng = np.random.default_rng(1)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-310, -1e-310, 1.0, -1.0, np.inf, -np.inf,
                        1.7976931348623157e308, -1.7976931348623157e308, 2.2250738585072014e-308])
    a = np.concatenate([np.repeat(special, len(special)), rng.standard_normal(20000) * 10.0 ** rng.uniform(-5, 5, 20000)])
    b = np.concatenate([np.tile(special, len(special)), rng.standard_normal(20000) * 10.0 ** rng.uniform(-5, 5, 20000)])
    b[-5000:] = a[-5000:]  # ties
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    out = torch.empty(len(a), dtype=torch.int32, device="cuda")
    fn = A.lib().amrh_selftest_order
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert fn(ad.data_ptr(), bd.data_ptr(), len(a), out.data_ptr()) == 0
    assert (out.cpu().numpy() == 31).all()
