"""GPU parity of the dual-energy formalism (section 2.2; the entropy per unit
volume as a passive scalar) against the oracle's step_dual: the scalar's
transport and the energy correction everywhere (xi huge), the hydro step
unchanged with xi = 0, and a cold Mach-800 flow with a transverse velocity
profile whose pressure only the formalism keeps; FP64 (relative L1 1e-12)
and the FP32 mode (1e-5)."""
import numpy as np
import pytest

import oracle
from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics
from test_gpu_uniform import rel_l1

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0
TOL = {A.AMR_FP64: 1e-12, A.AMR_FP32_ACC64: 1e-5}


def run(U0, S0, xi, steps, prec=A.AMR_FP64):
    from paper_1712_07070_b300.uniform import UniformGrid
    nz, ny, nx = U0.shape[1:]
    g = UniformGrid((nx, ny, nz), prec=prec, scheme={"dual_energy": 1, "dual_xi": xi})
    g.upload(U0)
    g.set_entropy(S0)
    dts = []
    for _ in range(steps):
        dt = g.min_dt()
        dts.append(dt)
        assert g.step(dt, count_unphysical=True) == 0
    out, S = g.download(), g.entropy()
    g.close()
    ref, Sr = U0, S0
    for dt in dts:
        ref, Sr, nbad = oracle.step_dual(ref, Sr, 1.0 / nx, dt, G53, xi)
        assert nbad == 0
    return out, S, ref, Sr


@pytest.mark.parametrize("prec", [A.AMR_FP64, A.AMR_FP32_ACC64])
def test_scalar_transport_and_energy_from_s(prec):
    U0 = ics.sod_noise(32, seed=13, ny=16, nz=48)
    S0 = oracle.entropy(U0, G53) * (1.0 + 0.05 * np.random.default_rng(2).random(U0.shape[1:]))
    out, S, ref, Sr = run(U0, S0, 1e300, 4, prec)
    assert (rel_l1(out, ref) <= TOL[prec]).all()
    assert np.abs(S - Sr).sum() <= TOL[prec] * np.abs(Sr).sum()


def test_xi_zero_is_the_plain_step_and_resets_s():
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.sod_noise(32, seed=14, ny=16, nz=48)
    out, S, ref, Sr = run(U0, oracle.entropy(U0, G53), 0.0, 3)
    g = UniformGrid((32, 16, 48))
    g.upload(U0)
    for _ in range(3):
        g.step(g.min_dt())
    plain = g.download()
    g.close()
    assert np.array_equal(out, plain)  # the hydro step of the dual-energy instance is bitwise the plain one
    assert np.abs(S - Sr).sum() <= 1e-12 * np.abs(Sr).sum()
    assert np.allclose(S, oracle.entropy(out, G53), rtol=1e-13, atol=0)


def test_cold_fast_shear_keeps_its_pressure():
    n = 64
    x = (np.arange(n) + 0.5) / n
    P0 = 1e-4
    U0 = np.zeros((5, 16, 16, n))
    U0[0] = 1.0
    U0[1] = 10.0
    U0[2] = 0.1 * np.sin(2 * np.pi * x)
    U0[4] = P0 / (G53 - 1) + 0.5 * (U0[1] ** 2 + U0[2] ** 2)
    out, S, ref, Sr = run(U0, oracle.entropy(U0, G53), 1e-2, 20)
    assert (rel_l1(out, ref) <= 1e-12).all()
    p = (G53 - 1) * (out[4] - 0.5 * (out[1] ** 2 + out[2] ** 2 + out[3] ** 2) / out[0])
    assert np.abs(p / P0 - 1).max() < 1e-4


@pytest.mark.parametrize("prec", [A.AMR_FP64, A.AMR_FP32_ACC64])
def test_box_batch_dual_energy(prec):
    """Dual energy in the box batch (one persistent launch per step, graph,
    per-box device dt): every box against the oracle's step_dual with the
    box's own Eq. (CFL2) step, the correction active everywhere (xi huge)
    and, on a cold fast shear box, at the default threshold."""
    from paper_1712_07070_b300.boxes import BoxBatch
    xi = 1e300
    B = BoxBatch(gamma=G53, prec=prec, scheme={"dual_energy": 1, "dual_xi": xi})
    sizes = [32, 16, 48]
    U0 = [ics.sod_noise(n, seed=20 + i) for i, n in enumerate(sizes)]
    S0 = [oracle.entropy(U, G53) * (1.0 + 0.05 * np.random.default_rng(i).random(U.shape[1:]))
          for i, U in enumerate(U0)]
    for U, S in zip(U0, S0):
        B.add_box(U, S)
    dts = B.advance(3).cpu().numpy()
    for i, n in enumerate(sizes):
        ref, Sr = U0[i], S0[i]
        for k in range(3):
            dt = oracle.dt_cfl2(ref, G53, 0.5, 1.0 / n)
            assert abs(dts[k, i] - dt) <= (1e-14 if prec == A.AMR_FP64 else 1e-6) * dt
            ref, Sr, nbad = oracle.step_dual(ref, Sr, 1.0 / n, dts[k, i], G53, xi)
            assert nbad == 0
        assert (rel_l1(B.download(i), ref) <= TOL[prec]).all(), n
        S = B.entropy(i)
        assert np.abs(S - Sr).sum() <= TOL[prec] * np.abs(Sr).sum(), n
    B.close()


def test_box_batch_dual_energy_requires_entropy_fields():
    from paper_1712_07070_b300.boxes import BoxBatch
    B = BoxBatch(gamma=G53, scheme={"dual_energy": 1})
    B.add_box(ics.sod_noise(16, seed=1))  # no entropy registered
    with pytest.raises(A.AmrHydroError):
        B.advance(1)
    B.close()


# ---- dual energy on refined hierarchies ----------------------------------------------------

def amr_compare_entropy(H, O, tol):
    """Every level's entropy against the oracle hierarchy's (relative L1)."""
    for l in range(H.lmax + 1):
        cg = H.corners(l)
        if not len(cg):
            continue
        S = H.entropy(l).cpu().numpy()
        num = den = 0.0
        for s, (x, y, z) in enumerate(cg.tolist()):
            r = O.lv[l].S[z:z + 8, y:y + 8, x:x + 8]
            num += np.abs(S[s] - r).sum()
            den += np.abs(r).sum()
        assert num <= tol * den, (l, num / den)


@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 1e-5)])
@pytest.mark.parametrize("xi,strong", [(1e-2, False), (1e300, True)])
def test_amr_dual_energy_matches_oracle(prec, tol, xi, strong):
    """The three-level W-cycle with the dual-energy formalism: the entropy's
    ghosts (interpolated with the conserved variables' positivity decision),
    its flux registers, fix-up, restriction and new-patch data against the
    oracle hierarchy; bit-exact patch lists, U and S of every level."""
    from oracle.amr import OracleHierarchy
    from paper_1712_07070_b300.amr import AmrHierarchy
    from test_gpu_amr import compare
    if strong:
        U0 = ics.blobs(32, seed=3)
        theta, nbuf = 0.05, (8, 4)
    else:
        U0 = ics.blobs(32, seed=5, contrast=10.0, mach=1.0)
        theta, nbuf = 0.3, (1, 1)
    S0 = oracle.entropy(U0, G53) * (1.0 + 0.05 * np.random.default_rng(4).random(U0.shape[1:]))
    H = AmrHierarchy(U0, lmax=2, theta=theta, nbuf=nbuf, prec=prec, max_patches=6000,
                     scheme={"dual_energy": 1, "dual_xi": xi}, S_root=S0)
    O = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=theta, nbuf=list(nbuf), S_root=S0, dual_xi=xi)
    assert H.n_patches(2) > 0
    for _ in range(2):
        H.advance_root()
        O.advance(0)
    compare(H, O, tol)
    amr_compare_entropy(H, O, tol)
    H.close()
