"""GPU parity of the other slope limiters and Riemann solvers (section 2.2:
HLLE, Roe, the exact solver)
against the oracle with the same scheme selected: uniform periodic steps in
FP64 (relative L1 <= 1e-12) and the FP32 mode (1e-5), the AMR W-cycle with
fix-up and regrid, and the batched-box launch; the adjoint refuses schemes
its hand-written reverse does not cover."""
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


def test_adjoint_refuses_other_schemes():
    import torch
    from paper_1712_07070_b300.uniform import UniformGrid
    g = UniformGrid((16, 16, 16), scheme=sch(A.AMR_LIM_GMINMOD, A.AMR_RS_HLLC, 1.5))
    U = g.state()
    lam = torch.zeros_like(U)
    with pytest.raises(A.AmrHydroError) as e:
        A.amr_hydro_step_adjoint(g.ctx, 0, 1e-3, U, lam, torch.empty_like(U))
    assert e.value.status == A.AMR_E_INVAL
    g.close()
