"""GPU parity of the other slope limiters and Riemann solvers (section 2.2:
HLLE, Roe, the exact solver) and of the VL scheme against the oracle with
the same scheme selected: uniform periodic steps in FP64 (relative L1 <=
1e-12) and the FP32 mode (1e-5), the AMR W-cycle with fix-up and regrid,
the batched-box launch and the host-buffer step; the adjoint refuses
schemes its hand-written reverse does not cover."""
import numpy as np
import pytest

import oracle
from oracle.amr import OracleHierarchy
from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics
from test_gpu_amr import compare
from test_gpu_uniform import PRECS, TOL, rel_l1

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0

SCHEMES = [
    (A.AMR_LIM_VANLEER, A.AMR_RS_HLLE, 1.5),
    (A.AMR_LIM_GMINMOD, A.AMR_RS_HLLC, 1.0),
    (A.AMR_LIM_GMINMOD, A.AMR_RS_HLLC, 1.5),
    (A.AMR_LIM_GMINMOD, A.AMR_RS_HLLE, 2.0),
    (A.AMR_LIM_ALBADA, A.AMR_RS_HLLC, 1.5),
    (A.AMR_LIM_ALBADA, A.AMR_RS_HLLE, 1.5),
    (A.AMR_LIM_VL_GMINMOD, A.AMR_RS_HLLC, 1.5),
    (A.AMR_LIM_VL_GMINMOD, A.AMR_RS_HLLE, 1.2),
    (A.AMR_LIM_VANLEER, A.AMR_RS_ROE, 1.5),
    (A.AMR_LIM_GMINMOD, A.AMR_RS_ROE, 2.0),
    (A.AMR_LIM_VANLEER, A.AMR_RS_EXACT, 1.5),
    (A.AMR_LIM_ALBADA, A.AMR_RS_EXACT, 1.5),
]


def sch(lim, rs, theta):
    return {"limiter": lim, "riemann": rs, "minmod_coeff": theta}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lim,rs,theta", SCHEMES)
def test_uniform_parity(prec, lim, rs, theta):
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.sod_noise(32, seed=11, ny=16, nz=48)  # non-cubic, several groups per axis
    nz, ny, nx = U0.shape[1:]
    g = UniformGrid((nx, ny, nz), prec=prec, scheme=sch(lim, rs, theta))
    g.upload(U0)
    dts = []
    for _ in range(4):
        dt = g.min_dt()
        dts.append(dt)
        g.step(dt)
    out = g.download()
    g.close()
    with oracle.scheme(lim, rs, theta):
        ref = U0
        for dt in dts:  # the oracle takes the GPU's dt sequence
            ref, nbad = oracle.step_periodic(ref, 1.0 / nx, dt, G53)
            assert nbad == 0
        odt = oracle.dt_cfl2(U0, G53, 0.5, 1.0 / nx)
    assert abs(dts[0] - odt) <= (1e-14 if prec == A.AMR_FP64 else 1e-6) * odt
    err = rel_l1(out, ref)
    assert (err <= TOL[prec]).all(), err


@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 1e-5)])
@pytest.mark.parametrize("theta,mild", [(1.5, False), (2.0, True)])
def test_amr_w_cycle_parity(prec, tol, theta, mild):
    # the MC limiter (theta = 2) with HLLE drives the Mach-2, contrast-100
    # blobs to negative pressure in the oracle too: milder blobs for it
    from paper_1712_07070_b300.amr import AmrHierarchy
    lim, rs = A.AMR_LIM_GMINMOD, A.AMR_RS_HLLE
    U0 = ics.blobs(32, seed=3, contrast=10.0, mach=1.0) if mild else ics.blobs(32, seed=3)
    with oracle.scheme(lim, rs, theta):
        H = AmrHierarchy(U0, lmax=2, theta=0.05, nbuf=(8, 4), prec=prec, max_patches=6000,
                         scheme=sch(lim, rs, theta))
        O = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8, 4])
        for _ in range(2):
            H.advance_root()
            O.advance(0)
        compare(H, O, tol)
    H.close()


@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 1e-5)])
@pytest.mark.parametrize("lim,rs", [(A.AMR_LIM_ALBADA, A.AMR_RS_HLLE), (A.AMR_LIM_VANLEER, A.AMR_RS_ROE)])
def test_boxes_parity(prec, tol, lim, rs):
    from paper_1712_07070_b300.boxes import BoxBatch
    theta = 1.5
    g14 = 1.4
    B = BoxBatch(gamma=g14, prec=prec, scheme=sch(lim, rs, theta))
    sizes = [32, 16, 48]
    U0 = [ics.kh_box(n, seed=40 + i, gamma=g14) for i, n in enumerate(sizes)]
    for U in U0:
        B.add_box(U)
    B.advance(3)
    with oracle.scheme(lim, rs, theta):
        for i, n in enumerate(sizes):
            ref, _ = oracle.run_periodic(U0[i], 1.0 / n, g14, 0.5, 3)
            err = rel_l1(B.download(i), ref)
            assert (err <= tol).all(), (n, err)
    B.close()


@pytest.mark.parametrize("scheme", [sch(A.AMR_LIM_GMINMOD, A.AMR_RS_HLLC, 1.5),
                                    dict(sch(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, 1.5), scheme=A.AMR_SCHEME_VL)])
def test_adjoint_refuses_other_schemes(scheme):
    import torch
    from paper_1712_07070_b300.uniform import UniformGrid
    g = UniformGrid((16, 16, 16), scheme=scheme)
    U = g.state()
    lam = torch.zeros_like(U)
    with pytest.raises(A.AmrHydroError) as e:
        A.amr_hydro_step_adjoint(g.ctx, 0, 1e-3, U, lam, torch.empty_like(U))
    assert e.value.status == A.AMR_E_INVAL
    g.close()


# ---- the VL scheme (section 2.2): a Riemann-solver half step, then the
# limited piecewise-linear states of U* without the Hancock increment
VL_SCHEMES = [
    (A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, 1.5),
    (A.AMR_LIM_GMINMOD, A.AMR_RS_HLLE, 1.5),
    (A.AMR_LIM_ALBADA, A.AMR_RS_ROE, 1.5),
    (A.AMR_LIM_VL_GMINMOD, A.AMR_RS_EXACT, 1.2),
]


def vl(lim, rs, theta):
    return dict(sch(lim, rs, theta), scheme=A.AMR_SCHEME_VL)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("lim,rs,theta", VL_SCHEMES)
def test_vl_uniform_parity(prec, lim, rs, theta):
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.sod_noise(32, seed=12, ny=48, nz=16)  # one group along z: the run wraps onto itself
    nz, ny, nx = U0.shape[1:]
    g = UniformGrid((nx, ny, nz), prec=prec, scheme=vl(lim, rs, theta))
    g.upload(U0)
    dts = []
    for _ in range(4):
        dt = g.min_dt()
        dts.append(dt)
        g.step(dt)
    out = g.download()
    g.close()
    with oracle.scheme(lim, rs, theta, vl=True):
        ref = U0
        for dt in dts:
            ref, nbad = oracle.step_periodic(ref, 1.0 / nx, dt, G53)
            assert nbad == 0
    err = rel_l1(out, ref)
    assert (err <= TOL[prec]).all(), err


@pytest.mark.parametrize("prec", PRECS)
def test_vl_turbulence_runs_parity(prec):
    """The VL launches on a level with z-runs of stacked groups (64^3: 4
    groups per z column) on the decaying-turbulence state."""
    from paper_1712_07070_b300.uniform import UniformGrid
    n = 64
    U0 = ics.turbulence(n, seed=5)
    g = UniformGrid((n, n, n), prec=prec, scheme=vl(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, 1.5))
    g.upload(U0)
    dt = g.min_dt()
    g.step(dt)
    g.step(dt)
    out = g.download()
    g.close()
    with oracle.scheme(vl=True):
        ref = U0
        for _ in range(2):
            ref, _ = oracle.step_periodic(ref, 1.0 / n, dt, G53)
    err = rel_l1(out, ref)
    assert (err <= TOL[prec]).all(), err


@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 1e-5)])
@pytest.mark.parametrize("lim,rs", [(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC), (A.AMR_LIM_GMINMOD, A.AMR_RS_ROE)])
def test_vl_boxes_parity(prec, tol, lim, rs):
    from paper_1712_07070_b300.boxes import BoxBatch
    g14 = 1.4
    B = BoxBatch(gamma=g14, prec=prec, scheme=vl(lim, rs, 1.5))
    sizes = [32, 16, 48]
    U0 = [ics.kh_box(n, seed=50 + i, gamma=g14) for i, n in enumerate(sizes)]
    for U in U0:
        B.add_box(U)
    B.advance(3)
    with oracle.scheme(lim, rs, 1.5, vl=True):
        for i, n in enumerate(sizes):
            ref, _ = oracle.run_periodic(U0[i], 1.0 / n, g14, 0.5, 3)
            err = rel_l1(B.download(i), ref)
            assert (err <= tol).all(), (n, err)
    B.close()


def pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nz", [16, 32, 80])
def test_vl_host_stream_bitwise(prec, nz):
    """The host-buffer step with the VL launches ordered by z-slab gives
    bitwise the device path's result (1, 2 and 5 slabs; CFL dt chained)."""
    from paper_1712_07070_b300.uniform import UniformGrid
    nx, ny = 32, 48
    U0 = ics.sod_noise(nx, seed=4, ny=ny, nz=nz)
    s = vl(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, 1.5)
    d = UniformGrid((nx, ny, nz), prec=prec, scheme=s)
    d.upload(U0)
    ref = []
    for _ in range(2):
        d.step(-1.0)
        ref.append(d.download())
    d.close()
    h = UniformGrid((nx, ny, nz), prec=prec, scheme=s)
    a, b = pinned(U0), pinned(np.zeros_like(U0))
    dt = -1.0
    for k in range(2):
        dt = h.step_host(a, b, dt)
        assert np.array_equal(b.numpy(), ref[k]), k
        a, b = b, a
    h.close()


def test_vl_full_size_512_sampled_cells():
    """One VL step of the 512^3 decaying-turbulence state on the device path:
    sampled cells recomputed by the oracle on their periodic 9^3
    neighbourhood (the VL step's domain of dependence is +-3 cells)."""
    from paper_1712_07070_b300.uniform import UniformGrid
    from test_gpu_uniform import subcube
    n = 512
    U0 = ics.turbulence(n, seed=1)
    g = UniformGrid((n, n, n), scheme=vl(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, 1.5))
    g.upload(U0)
    dt = g.min_dt()
    g.step(dt)
    out = g.download()
    g.close()
    rng = np.random.default_rng(8)
    cells = rng.integers(0, n, size=(24, 3))
    cells[:3] = [[0, 0, 0], [n - 1, n - 1, n - 1], [15, 16, 31]]
    with oracle.scheme(vl=True):
        for c in cells:
            r, _ = oracle.step_periodic(subcube(U0, c, 4), 1.0 / n, dt, G53)
            scale = np.abs(U0[:, c[2], c[1], c[0]]).max()
            assert np.abs(out[:, c[2], c[1], c[0]] - r[:, 4, 4, 4]).max() <= 1e-12 * scale, c


# ---- the VL scheme on refined hierarchies ------------------------------------------------

def vl_sch(lim, rs, theta=1.5):
    return dict(sch(lim, rs, theta), scheme=A.AMR_SCHEME_VL)


@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 1e-5)])
@pytest.mark.parametrize("lim,rs,mild", [(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, False),
                                         (A.AMR_LIM_GMINMOD, A.AMR_RS_HLLE, True)])
def test_vl_amr_w_cycle_parity(prec, tol, lim, rs, mild):
    """VL on the three-level blob hierarchy: the corrector of groups next to
    coarse-fine interfaces reads the half step of their ghost cells, made
    from the interpolated U^n three cells deep; bit-exact patch lists and
    every level's cells against the oracle hierarchy with VL selected."""
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(32, seed=3, contrast=10.0, mach=1.0) if mild else ics.blobs(32, seed=3)
    with oracle.scheme(lim, rs, 1.5, vl=True):
        H = AmrHierarchy(U0, lmax=2, theta=0.05, nbuf=(8, 4), prec=prec, max_patches=6000,
                         scheme=vl_sch(lim, rs))
        O = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8, 4])
        assert H.n_patches(2) > 0
        for _ in range(2):
            H.advance_root()
            O.advance(0)
        compare(H, O, tol)
    H.close()


def test_vl_amr_interfaces_and_conservation():
    """Many coarse-fine interfaces (small flag buffer): parity with the oracle
    and the composite conserved sums across fix-up and regrid."""
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(32, seed=5, contrast=10.0, mach=1.0)
    with oracle.scheme(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC, 1.5, vl=True):
        H = AmrHierarchy(U0, lmax=2, theta=0.3, nbuf=(1, 1), max_patches=6000,
                         scheme=vl_sch(A.AMR_LIM_VANLEER, A.AMR_RS_HLLC))
        O = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1, 1])
        assert 0 < H.n_patches(1) < 8 * 64
        s0 = H.conserved_total()
        for _ in range(2):
            H.advance_root()
            O.advance(0)
        compare(H, O, 1e-12)
        s1 = H.conserved_total()
    scale = np.abs(U0).reshape(5, -1).sum(1) / 32 ** 3
    assert (np.abs(s1 - s0) <= 1e-13 * scale).all(), (s1 - s0) / scale
    H.close()
