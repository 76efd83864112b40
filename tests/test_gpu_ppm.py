"""GPU parity of PPM reconstruction (section 2.2, Colella & Woodward 1984;
three ghost cells) with the MUSCL-Hancock and CTU schemes against the
oracle: uniform periodic steps (FP64 relative L1 <= 1e-12; the FP32 mode
1e-5 for MUSCL-Hancock, 5e-5 for CTU), levels with z-runs, the AMR W-cycle
(ghost patches interpolated three cells deep), the batched boxes, the
host-buffer step (bitwise against the device path), and sampled cells of a
512^3 step."""
import numpy as np
import pytest

import oracle
from oracle.amr import OracleHierarchy
from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics
from test_gpu_amr import compare
from test_gpu_uniform import PRECS, rel_l1

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0
MH, CTU = A.AMR_SCHEME_MH, A.AMR_SCHEME_CTU
# the CTU bound of the FP32 mode is derived in test_gpu_ctu.py
TOL = {(MH, A.AMR_FP64): 1e-12, (MH, A.AMR_FP32_ACC64): 1e-5,
       (CTU, A.AMR_FP64): 1e-12, (CTU, A.AMR_FP32_ACC64): 5e-5}


def ppm(scheme, lim=A.AMR_LIM_VANLEER, rs=A.AMR_RS_HLLC, theta=1.5):
    return {"limiter": lim, "riemann": rs, "minmod_coeff": theta, "scheme": scheme, "recon": A.AMR_RECON_PPM}


def oscheme(scheme, lim=A.AMR_LIM_VANLEER, rs=A.AMR_RS_HLLC, theta=1.5):
    return oracle.scheme(lim, rs, theta, ctu=scheme == CTU, ppm=True)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("scheme", [MH, CTU])
@pytest.mark.parametrize("lim,rs,theta", [(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, 1.5),
                                          (A.AMR_LIM_GMINMOD, A.AMR_RS_ROE, 2.0),
                                          (A.AMR_LIM_ALBADA, A.AMR_RS_HLLE, 1.5)])
def test_uniform_parity(prec, scheme, lim, rs, theta):
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.sod_noise(32, seed=31, ny=16, nz=48)
    nz, ny, nx = U0.shape[1:]
    g = UniformGrid((nx, ny, nz), prec=prec, scheme=ppm(scheme, lim, rs, theta))
    g.upload(U0)
    dts = []
    for _ in range(4):
        dt = g.min_dt()
        dts.append(dt)
        g.step(dt)
    out = g.download()
    g.close()
    with oscheme(scheme, lim, rs, theta):
        ref = U0
        for dt in dts:
            ref, nbad = oracle.step_periodic(ref, 1.0 / nx, dt, G53)
            assert nbad == 0
    err = rel_l1(out, ref)
    assert (err <= TOL[scheme, prec]).all(), err


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("scheme", [MH, CTU])
def test_turbulence_runs_parity(prec, scheme):
    from paper_1712_07070_b300.uniform import UniformGrid
    n = 64
    U0 = ics.turbulence(n, seed=7)
    g = UniformGrid((n, n, n), prec=prec, scheme=ppm(scheme))
    g.upload(U0)
    for _ in range(2):
        g.step(-1.0)
    out = g.download()
    g.close()
    with oscheme(scheme):
        ref, _ = oracle.run_periodic(U0, 1.0 / n, G53, 0.5, 2)
    err = rel_l1(out, ref)
    assert (err <= TOL[scheme, prec]).all(), err


@pytest.mark.parametrize("scheme", [MH, CTU])
def test_long_columns_z_runs_parity(scheme):
    """64 x 64 x 512: 512 groups in 16 columns of 32, more than one CTA round,
    so the step marches z-runs of several groups (the next group's tables are
    loaded while the march stages the current group's planes)."""
    from paper_1712_07070_b300.uniform import UniformGrid
    nx, ny, nz = 64, 64, 512
    U0 = ics.sod_noise(nx, seed=12, ny=ny, nz=nz)
    g = UniformGrid((nx, ny, nz), scheme=ppm(scheme))
    g.upload(U0)
    dt = g.min_dt()
    g.step(dt)
    out = g.download()
    g.close()
    with oscheme(scheme):
        ref, nbad = oracle.step_periodic(U0, 1.0 / nx, dt, G53)
    assert nbad == 0
    err = rel_l1(out, ref)
    assert (err <= 1e-12).all(), err


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("scheme", [MH, CTU])
def test_amr_w_cycle_parity(prec, scheme):
    from paper_1712_07070_b300.amr import AmrHierarchy
    # at contrast 100 and Mach 2 PPM drives the oracle itself to negative pressure
    U0 = ics.blobs(32, seed=3, contrast=30.0, mach=1.5)
    with oscheme(scheme):
        H = AmrHierarchy(U0, lmax=2, theta=0.05, nbuf=(8, 4), prec=prec, max_patches=6000, scheme=ppm(scheme))
        O = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8, 4])
        for _ in range(2):
            H.advance_root()
            O.advance(0)
        compare(H, O, TOL[scheme, prec])
    H.close()


@pytest.mark.parametrize("prec", PRECS)
def test_boxes_parity(prec):
    from paper_1712_07070_b300.boxes import BoxBatch
    g14 = 1.4
    B = BoxBatch(gamma=g14, prec=prec, scheme=ppm(MH))
    sizes = [32, 16, 48]
    U0 = [ics.kh_box(n, seed=70 + i, gamma=g14) for i, n in enumerate(sizes)]
    for U in U0:
        B.add_box(U)
    B.advance(3)
    with oscheme(MH):
        for i, n in enumerate(sizes):
            ref, _ = oracle.run_periodic(U0[i], 1.0 / n, g14, 0.5, 3)
            err = rel_l1(B.download(i), ref)
            assert (err <= TOL[MH, prec]).all(), (n, err)
    B.close()


def pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("scheme", [MH, CTU])
def test_host_stream_bitwise(scheme):
    from paper_1712_07070_b300.uniform import UniformGrid
    nx, ny, nz = 32, 48, 64
    U0 = ics.sod_noise(nx, seed=10, ny=ny, nz=nz)
    d = UniformGrid((nx, ny, nz), scheme=ppm(scheme))
    d.upload(U0)
    ref = []
    for _ in range(2):
        d.step(-1.0)
        ref.append(d.download())
    d.close()
    h = UniformGrid((nx, ny, nz), scheme=ppm(scheme))
    a, b = pinned(U0), pinned(np.zeros_like(U0))
    dt = -1.0
    for k in range(2):
        dt = h.step_host(a, b, dt)
        assert np.array_equal(b.numpy(), ref[k]), k
        a, b = b, a
    h.close()


@pytest.mark.parametrize("scheme", [MH, CTU])
def test_full_size_512_sampled_cells(scheme):
    """One step of the 512^3 decaying-turbulence state: sampled cells
    recomputed by the oracle on their periodic 9^3 neighbourhood (the domain
    of dependence of a PPM step is +-3 cells)."""
    from paper_1712_07070_b300.uniform import UniformGrid
    from test_gpu_uniform import subcube
    n = 512
    U0 = ics.turbulence(n, seed=1)
    g = UniformGrid((n, n, n), scheme=ppm(scheme))
    g.upload(U0)
    dt = g.min_dt()
    g.step(dt)
    out = g.download()
    g.close()
    rng = np.random.default_rng(11)
    cells = rng.integers(0, n, size=(16, 3))
    cells[:3] = [[0, 0, 0], [n - 1, n - 1, n - 1], [17, 14, 31]]
    with oscheme(scheme):
        for c in cells:
            r, _ = oracle.step_periodic(subcube(U0, c, 4), 1.0 / n, dt, G53)
            scale = np.abs(U0[:, c[2], c[1], c[0]]).max()
            assert np.abs(out[:, c[2], c[1], c[0]] - r[:, 4, 4, 4]).max() <= 1e-12 * scale, c
