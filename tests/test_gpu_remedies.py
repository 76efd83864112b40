"""GPU parity of the remedies for unphysical results (section 2.2) against
the oracle with the same remedies: the Roe solver's intermediate-state check
on a double-rarefaction tube, the first-order cell remedies on the Mach-2,
contrast-100 blobs (which drive the plain step to negative pressure), the
split remedy (CTU at Courant number 1), the level retry with dt x 0.8, the
AMR W-cycle with CTU on the blobs, the FP32 mode and the host-buffer step."""
import numpy as np
import pytest

import oracle
from oracle.amr import OracleHierarchy
from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics
from test_gpu_amr import compare
from test_gpu_uniform import rel_l1

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0


def run_pair(U0, scheme, okw, steps, cfl=0.5, prec=A.AMR_FP64):
    """GPU steps with the host-read dt of each step, and the oracle on the
    same dt sequence; returns (gpu state, oracle state, oracle remedy counts)."""
    from paper_1712_07070_b300.uniform import UniformGrid
    nz, ny, nx = U0.shape[1:]
    g = UniformGrid((nx, ny, nz), prec=prec, cfl=cfl, scheme=scheme)
    g.upload(U0)
    dts = []
    for _ in range(steps):
        dt = g.min_dt()
        dts.append(dt)
        assert g.step(dt, count_unphysical=True) == 0
    out = g.download()
    g.close()
    with oracle.scheme(fallback=True, **okw):
        oracle.fallback_counts()
        ref = U0
        for dt in dts:
            ref, nbad = oracle.step_periodic(ref, 1.0 / nx, dt, G53)
            assert nbad == 0
        counts = oracle.fallback_counts()
    return out, ref, counts


def test_roe_intermediate_state_check():
    U0 = ics.riemann_tube(32, (1.0, -2.0, 0.1), (1.0, 2.0, 0.1), axis=0, transverse=16, gamma=G53)
    out, ref, _ = run_pair(U0, {"riemann": A.AMR_RS_ROE, "fallback": 1}, {"riemann": oracle.RS_ROE}, 4)
    assert (rel_l1(out, ref) <= 1e-12).all()


def test_cell_remedies_on_blobs():
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.blobs(32, seed=3)
    g = UniformGrid((32, 32, 32))  # without the remedies the second step leaves bad cells
    g.upload(U0)
    bad = [g.step(-1.0, count_unphysical=True) for _ in range(2)]
    g.close()
    # (the plain step's count depends on how a face state with negative
    # pressure propagates NaN, which only the remedies define: 9 in the
    # oracle, fewer through the device's bit-pattern sign tests)
    assert bad[0] == 0 and bad[1] > 0
    out, ref, counts = run_pair(U0, {"fallback": 1}, {}, 4)
    assert counts[0] > 0  # the unsplit first-order remedy ran
    assert (rel_l1(out, ref) <= 1e-12).all()


def test_split_remedy_ctu_courant_1():
    U0 = ics.blobs(32, seed=3)
    out, ref, counts = run_pair(U0, {"scheme": A.AMR_SCHEME_CTU, "fallback": 1}, {"ctu": True}, 4, cfl=1.0)
    assert counts[1] > 0  # the split remedy ran
    assert (rel_l1(out, ref) <= 1e-12).all()


def test_level_retry_dt_x_0_8():
    from paper_1712_07070_b300.uniform import UniformGrid
    n = 32
    U0 = ics.blobs(n, seed=3)
    cfl = 1.3
    with oracle.scheme(fallback=True, ctu=True):  # advance to the first step that needs a retry
        for _ in range(6):
            dt = oracle.dt_cfl(U0, G53, cfl, 1 / n)
            _, nbad = oracle.step_periodic(U0, 1 / n, dt, G53)
            if nbad:
                break
            U0, _ = oracle.step_periodic(U0, 1 / n, dt, G53)
        assert nbad
        ref, taken = oracle.step_retry(U0, 1 / n, dt, G53, dt_min=1e-4 * dt)
    g = UniformGrid((n, n, n), cfl=cfl, scheme={"scheme": A.AMR_SCHEME_CTU, "fallback": 1, "dt_min": 1e-4 * dt})
    g.upload(U0)
    t0 = g.time()
    g.step(-1.0)  # the device's Eq. CFL1 dt, then the retries
    assert g.time() - t0 == pytest.approx(taken, rel=1e-13)
    out = g.download()
    g.close()
    assert (rel_l1(out, ref) <= 1e-12).all()
    g = UniformGrid((n, n, n), cfl=cfl, scheme={"scheme": A.AMR_SCHEME_CTU, "fallback": 1, "dt_min": 0.9 * dt})
    g.upload(U0)
    with pytest.raises(A.AmrHydroError) as e:  # dt x 0.8 would fall below dt_min
        g.step(dt)
    assert e.value.status == A.AMR_E_UNPHYSICAL
    assert g.time() == t0  # the level keeps U^n and its time
    g.close()


def test_amr_ctu_blobs_with_remedies():
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(32, seed=3)  # contrast 100, Mach 2: the plain CTU oracle goes unphysical
    sch = {"scheme": A.AMR_SCHEME_CTU, "fallback": 1}
    with oracle.scheme(ctu=True, fallback=True):
        H = AmrHierarchy(U0, lmax=2, theta=0.05, nbuf=(8, 4), max_patches=6000, scheme=sch)
        O = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8, 4])
        for _ in range(2):
            H.advance_root()
            O.advance(0)
        compare(H, O, 1e-12)
    H.close()


def test_fp32_mode_stays_physical():
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.blobs(32, seed=3)
    g = UniformGrid((32, 32, 32), prec=A.AMR_FP32_ACC64, scheme={"fallback": 1})
    g.upload(U0)
    for _ in range(6):
        assert g.step(-1.0, count_unphysical=True) == 0
    g.close()


def test_host_stream_bitwise_with_remedies():
    import torch
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.blobs(32, seed=3)
    d = UniformGrid((32, 32, 32), scheme={"fallback": 1})
    d.upload(U0)
    ref = []
    for _ in range(3):
        d.step(-1.0)
        ref.append(d.download())
    d.close()
    h = UniformGrid((32, 32, 32), scheme={"fallback": 1})
    a = torch.from_numpy(np.ascontiguousarray(U0)).pin_memory()
    b = torch.zeros_like(a).pin_memory()
    dt = -1.0
    for k in range(3):
        dt = h.step_host(a, b, dt)
        assert np.array_equal(b.numpy(), ref[k]), k
        a, b = b, a
    h.close()
