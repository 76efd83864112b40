"""amr_hydro_advance_host: the uniform step from a host state to a host state
with the copies overlapped by z-slabs must give bitwise the results of the
device path (upload, amr_hydro_advance_level, download), for a given dt, for
the CFL dt of the input, chained through the returned dt, and in place; it
rejects a level that is not the whole root grid in the uniform order; at the
benchmark's 512^3 size, sampled cells match the oracle."""
import numpy as np
import pytest

import oracle
from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics
from paper_1712_07070_b300.uniform import UniformGrid

pytestmark = pytest.mark.gpu
PRECS = [A.AMR_FP64, A.AMR_FP32_ACC64]


def pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def device_steps(U0, prec, dts):
    """Reference: upload once, then one device step per dt (dt < 0: device
    CFL dt); returns the state after each step."""
    nz, ny, nx = U0.shape[1:]
    g = UniformGrid((nx, ny, nz), prec=prec)
    g.upload(U0)
    out = []
    for dt in dts:
        g.step(dt)
        out.append(g.download())
    mdt = g.min_dt()
    g.close()
    return out, mdt


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(32, 48, 64), (64, 64, 64)])
def test_fixed_dt_bitwise(prec, shape):
    nx, ny, nz = shape
    U0 = ics.sod_noise(nx, seed=7, ny=ny, nz=nz)
    ref, _ = device_steps(U0, prec, [2e-3])
    g = UniformGrid(shape, prec=prec)
    hin, hout = pinned(U0), pinned(np.zeros_like(U0))
    g.step_host(hin, hout, 2e-3)
    assert np.array_equal(hout.numpy(), ref[0])
    assert g.time() == pytest.approx(2e-3, rel=0, abs=0)
    g.close()


@pytest.mark.parametrize("prec", PRECS)
def test_cfl_dt_chained_and_dt_next(prec):
    U0 = ics.turbulence(32, seed=3)
    ref, ref_dt = device_steps(U0, prec, [-1.0, -1.0, -1.0])
    g = UniformGrid((32, 32, 32), prec=prec)
    a, b = pinned(U0), pinned(np.zeros_like(U0))
    dt = -1.0
    for k in range(3):
        dt = g.step_host(a, b, dt)
        assert np.array_equal(b.numpy(), ref[k]), k
        a, b = b, a
    assert dt == ref_dt  # CFL dt of the last output, as the device computes it
    assert dt == g.min_dt()
    g.close()


def test_in_place_and_pageable():
    U0 = ics.sod_noise(32, seed=2)
    ref, _ = device_steps(U0, A.AMR_FP64, [1e-3])
    g = UniformGrid((32, 32, 32))
    buf = pinned(U0)
    g.step_host(buf, buf, 1e-3)  # U_out == U_in
    assert np.array_equal(buf.numpy(), ref[0])
    src, dst = np.ascontiguousarray(U0), np.zeros_like(U0)  # pageable numpy arrays
    g2 = UniformGrid((32, 32, 32))
    g2.step_host(src, dst, 1e-3)
    assert np.array_equal(dst, ref[0])
    g.close()
    g2.close()


def test_rejects_non_uniform_order():
    import torch
    n = 32
    p = A.make_params(root_n=(n, n, n))
    ctx = A.amr_hydro_init(p, None)
    corner, sib, parent, child = A.amr_hydro_uniform_tables((n // 8,) * 3)
    # swap the first two groups: a valid level, but not the uniform slot order
    perm = np.arange(len(corner))
    perm[:8], perm[8:16] = np.arange(8, 16), np.arange(8)
    inv = np.argsort(perm)
    corner = corner[perm]
    sib = np.where(sib[perm] >= 0, inv[np.maximum(sib[perm], 0)], -1).astype(np.int32)
    t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (corner, sib, parent, child)]
    U = [torch.zeros((len(corner), 5, 8, 8, 8), dtype=torch.float64, device="cuda") for _ in range(2)]
    A.amr_hydro_set_level(ctx, 0, len(corner), U[0], U[1], *t, t=0.0)
    hin = pinned(ics.uniform_state(n))
    with pytest.raises(A.AmrHydroError) as e:
        A.amr_hydro_advance_host(ctx, hin, pinned(np.zeros(hin.shape)), 1e-3)
    assert e.value.status == A.AMR_E_INVAL
    A.amr_hydro_destroy(ctx)


def test_full_size_512_host_stream_sampled_cells():
    """The end-to-end path of the benchmark (512^3 turbulence, host buffers,
    z-slab overlap) in its launch configuration: 32 sampled cells of the
    host result recomputed one by one by the oracle on their periodic 9^3
    neighbourhood (the step's domain of dependence is +-2 cells)."""
    from test_gpu_uniform import subcube
    n = 512
    U0 = ics.turbulence(n, seed=1)
    dt = oracle.dt_cfl2(U0, 5.0 / 3.0, 0.5, 1.0 / n)
    g = UniformGrid((n, n, n))
    a, b = pinned(U0), pinned(np.empty_like(U0))
    dt_next = g.step_host(a, b, dt)
    assert dt_next > 0
    out = b.numpy()
    rng = np.random.default_rng(3)
    cells = rng.integers(0, n, size=(32, 3))
    cells[:4] = [[0, 0, 0], [n - 1, n - 1, n - 1], [5, 9, 15], [100, 200, 16]]  # incl. slab boundaries
    for c in cells:
        r, _ = oracle.step_periodic(subcube(U0, c, 4), 1.0 / n, dt, 5.0 / 3.0)
        scale = np.abs(U0[:, c[2], c[1], c[0]]).max()
        assert np.abs(out[:, c[2], c[1], c[0]] - r[:, 4, 4, 4]).max() <= 1e-12 * scale, c
    g.close()
