"""Pins of the oracle's remedies for unphysical results (section 2.2 lists
them; the readings are in the oracle's header):

  * (i) the Roe solver's intermediate states: on a double rarefaction whose
    linearised intermediate density is negative the face takes exactly the
    HLLE flux; on a Sod face the Roe flux is unchanged; a tube that fails
    with plain Roe runs clean with the check;
  * (0) with the remedies on, a face with an unphysical state has no flux,
    so the cells on both sides take the cell remedies;
  * (ii) a cell left unphysical by the step is replaced by the first-order
    unsplit update of U^n, written out here face by face with the pinned
    Riemann solvers; every other cell is bitwise the plain step's;
  * (iii) where (ii) is unphysical too, the first-order split update (x, y,
    then z sweeps over the cell's 3x3x3 neighbourhood), written out here;
  * (iv)-(v) the retry loop takes dt x 0.8^k and its result is the plain
    step at that dt;
  * the Mach-2, contrast-100 blobs, which drive every scheme to negative
    pressure within a few steps, stay physical with the remedies.
"""
import numpy as np
import pytest

import oracle
from paper_1712_07070_b300 import ics

G53 = 5.0 / 3.0


def physical(u):
    w = oracle.prim(u, G53)
    return w[0] > 0 and w[4] > 0


def test_roe_intermediate_state_check():
    uL = oracle.cons([1.0, -2.0, 0.0, 0.0, 0.1], G53)
    uR = oracle.cons([1.0, 2.0, 0.0, 0.0, 0.1], G53)
    # Roe's linearised left intermediate density: rho_L + a1 with
    # a1 = (dp - rho~ a~ du)/(2 a~^2); here dp = 0, rho~ = 1, du = 4 -> a1 = -2/a~ < -1
    plain = oracle.roe(uL, uR, 0, G53)
    with oracle.scheme(riemann=oracle.RS_ROE, fallback=True):
        checked = oracle.roe(uL, uR, 0, G53)
    assert np.array_equal(checked, oracle.hlle(uL, uR, 0, G53))
    assert not np.array_equal(checked, plain)
    sL = oracle.cons([1.0, 0.0, 0.0, 0.0, 1.0], G53)
    sR = oracle.cons([0.125, 0.0, 0.0, 0.0, 0.1], G53)
    with oracle.scheme(riemann=oracle.RS_ROE, fallback=True):
        same = oracle.roe(sL, sR, 0, G53)
    assert np.array_equal(same, oracle.roe(sL, sR, 0, G53))


def test_roe_check_keeps_a_rarefaction_tube_physical():
    U = ics.riemann_tube(32, (1.0, -2.0, 0.1), (1.0, 2.0, 0.1), axis=0, gamma=G53)
    with oracle.scheme(riemann=oracle.RS_ROE):
        _, nbad = oracle.step_periodic(U, 1 / 32, oracle.dt_cfl(U, G53, 0.5, 1 / 32), G53)
    assert nbad > 0
    with oracle.scheme(riemann=oracle.RS_ROE, fallback=True):
        V = U
        for _ in range(6):
            V, nbad = oracle.step_periodic(V, 1 / 32, oracle.dt_cfl(V, G53, 0.5, 1 / 32), G53)
            assert nbad == 0


def cell(U, x, y, z):
    n = U.shape[1:]
    return U[:, z % n[0], y % n[1], x % n[2]].copy()


def first_order_unsplit(U, c, r):
    x, y, z = c
    u0 = cell(U, x, y, z)
    div = np.zeros(5)
    for d, e in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
        up = cell(U, x + e[0], y + e[1], z + e[2])
        um = cell(U, x - e[0], y - e[1], z - e[2])
        div += oracle.hllc(u0, up, d, G53) - oracle.hllc(um, u0, d, G53)
    return u0 - r * div


def sweep(vm, v0, vp, d, r):
    return v0 - r * (oracle.hllc(v0, vp, d, G53) - oracle.hllc(vm, v0, d, G53))


def first_order_split(U, c, r):
    x, y, z = c
    X = {(j, k): sweep(cell(U, x - 1, y + j, z + k), cell(U, x, y + j, z + k), cell(U, x + 1, y + j, z + k), 0, r)
         for j in (-1, 0, 1) for k in (-1, 0, 1)}
    Y = {k: sweep(X[-1, k], X[0, k], X[1, k], 1, r) for k in (-1, 0, 1)}
    return sweep(Y[-1], Y[0], Y[1], 2, r)


def first_bad_step(U, n, cfl, kw, max_steps=6):
    """Advance with the remedies until the plain step would leave unphysical
    cells; returns (state, dt) of that step."""
    for _ in range(max_steps):
        with oracle.scheme(**kw):
            dt = oracle.dt_cfl(U, G53, cfl, 1 / n)
            _, nbad = oracle.step_periodic(U, 1 / n, dt, G53)
        if nbad:
            return U, dt
        with oracle.scheme(fallback=True, **kw):
            U, _ = oracle.step_periodic(U, 1 / n, dt, G53)
    raise AssertionError("no unphysical step")


@pytest.mark.parametrize("cfl,kw,which", [(0.5, {}, 0), (1.0, {"ctu": True}, 1)])
def test_cell_remedies_are_the_first_order_updates(cfl, kw, which):
    n = 32
    U, dt = first_bad_step(ics.blobs(n, seed=3), n, cfl, kw)
    with oracle.scheme(**kw):
        A, _ = oracle.step_periodic(U, 1 / n, dt, G53)
    with oracle.scheme(fallback=True, **kw):
        oracle.fallback_counts()
        B, nbad = oracle.step_periodic(U, 1 / n, dt, G53)
        counts = oracle.fallback_counts()
    assert nbad == 0 and counts[2] == 0 and counts[which] > 0, counts
    # the remedied cells: those of the plain step's unphysical cells and the
    # cells next to a face with an unphysical state (no flux with the
    # remedies on); every other cell is bitwise the plain step's
    same = np.all((A == B) | (np.isnan(A) & np.isnan(B)), axis=0)
    bad = [(x, y, z) for z, y, x in np.argwhere(~same)]
    assert len(bad) == counts[0] + counts[1]
    assert all(not physical(A[:, z, y, x]) for x, y, z in bad if not np.isfinite(A[:, z, y, x]).all())
    r = dt / (1 / n)
    n_split = 0
    for c in bad:
        x, y, z = c
        u = first_order_unsplit(U, c, r)
        if not physical(u):
            u = first_order_split(U, c, r)
            n_split += 1
        assert np.allclose(B[:, z, y, x], u, rtol=1e-13, atol=1e-14 * np.abs(u).max()), c
    assert n_split == counts[1]


def test_retry_driver_takes_dt_times_0_8_powers():
    n = 32
    U, dt = first_bad_step(ics.blobs(n, seed=3), n, 1.3, {"ctu": True})
    with oracle.scheme(fallback=True, ctu=True):
        _, nbad = oracle.step_periodic(U, 1 / n, dt, G53)
        assert nbad > 0  # the cell remedies are not enough at this dt
        V, taken = oracle.step_retry(U, 1 / n, dt, G53, dt_min=1e-3 * dt)
        k = round(np.log(taken / dt) / np.log(0.8))
        assert k >= 1 and taken == pytest.approx(dt * 0.8 ** k, rel=1e-15)
        W, nbad2 = oracle.step_periodic(U, 1 / n, taken, G53)
        assert nbad2 == 0 and np.array_equal(V, W)
        with pytest.raises(FloatingPointError):
            oracle.step_retry(U, 1 / n, dt, G53, dt_min=0.9 * dt)


@pytest.mark.parametrize("kw", [{}, {"ppm": True}, {"ctu": True}, {"ctu": True, "ppm": True}])
def test_blobs_stay_physical_with_the_remedies(kw):
    n = 32
    U = ics.blobs(n, seed=3)
    with oracle.scheme(fallback=True, **kw):
        for _ in range(6):
            U, nbad = oracle.step_periodic(U, 1 / n, oracle.dt_cfl(U, G53, 0.5, 1 / n), G53)
            assert nbad == 0


@pytest.mark.parametrize("name", ["hllc", "hlle", "roe", "exact_flux"])
def test_a_face_with_an_unphysical_state_has_no_flux(name):
    """With the remedies on, every solver returns NaN for a face whose left or
    right state has rho <= 0 or P <= 0 (so both cells count as unphysical),
    and a finite flux for physical states."""
    good = oracle.cons([1.0, 0.1, 0.0, 0.0, 1.0], G53)
    neg_p = good.copy()
    neg_p[4] = 0.5 * good[1] ** 2 / good[0] - 0.01  # E below the kinetic energy: P < 0
    neg_rho = good.copy()
    neg_rho[0] = -0.1
    fn = getattr(oracle, name)
    with oracle.scheme(fallback=True):
        assert np.isfinite(fn(good, good, 0, G53)).all()
        for bad in (neg_p, neg_rho):
            assert np.isnan(fn(good, bad, 1, G53)).all()
            assert np.isnan(fn(bad, good, 2, G53)).all()
