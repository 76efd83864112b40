"""Pins of the FP64 CPU oracle against facts fixed by the mathematics and by
published closed forms -- never against the oracle itself.

Each pin is chosen so that a plausible slip in the oracle fails it:
  * exact Riemann solver: Newton vs bisection, and the textbook Sod star state
    (Toro 2009, Table 4.2, test 1: p* = 0.30313, u* = 0.92745);
  * HLLC (section 2.2): consistency F(U,U)=F(U), exact stationary contact,
    exact upwinding for supersonic states, mirror antisymmetry;
  * the whole MUSCL-Hancock step (section 2.2): Sod tube converging to the
    exact solution, uniform states unchanged to the bit, conservation to
    round-off, mirror and axis-permutation symmetry, second-order
    convergence on a smooth advected wave (fails if the Hancock half step,
    the slopes or a flux sign is dropped);
  * Eq. CFL2 of section 2.6 against a hand-evaluated cell.
"""
import numpy as np
import pytest

import oracle
from paper_1712_07070_b300 import ics

G53 = 5.0 / 3.0


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


# ---- exact Riemann solver ------------------------------------------------------

def test_exact_riemann_newton_matches_bisection():
    cases = [
        ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4),       # Sod
        ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4), 1.4),        # 123 problem (two rarefactions)
        ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 1.4),     # strong blast
        ((5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.0950), 1.4),  # two shocks
        ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), G53),
    ]
    for L, R, g in cases:
        ps, _ = oracle.exact_star(*L, *R, g)
        pb = oracle.exact_pstar_bisect(*L, *R, g)
        assert abs(ps - pb) <= 1e-13 * pb, (L, R, ps, pb)


def test_exact_riemann_sod_textbook_star_state():
    # Toro (2009), Table 4.2, test 1 (Sod, gamma=1.4): p* = 0.30313, u* = 0.92745
    ps, us = oracle.exact_star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert abs(ps - 0.30313) < 5e-6
    assert abs(us - 0.92745) < 5e-6


def test_exact_riemann_sample_jump_conditions():
    # across the right-moving shock of Sod the Rankine-Hugoniot mass flux
    # rho (u - S) is continuous; far states reproduce the data
    g = 1.4
    r, u, p = oracle.exact_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, [-5.0, 5.0])
    assert np.allclose(r, [1.0, 0.125]) and np.allclose(p, [1.0, 0.1]) and np.allclose(u, 0.0)
    ps, us = oracle.exact_star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g)
    cR = np.sqrt(g * 0.1 / 0.125)
    S = cR * np.sqrt((g + 1) / (2 * g) * ps / 0.1 + (g - 1) / (2 * g))
    r2, u2, p2 = oracle.exact_sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), g, [S - 1e-9])
    assert abs(r2[0] * (u2[0] - S) - 0.125 * (0.0 - S)) < 1e-9


# ---- HLLC ------------------------------------------------------------------------

def random_state(rng, g):
    rho = rng.uniform(0.2, 3.0)
    v = rng.normal(0, 1.0, 3)
    P = rng.uniform(0.1, 3.0)
    return oracle.cons([rho, *v, P], g)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_consistency(d):
    rng = np.random.default_rng(10 + d)
    for _ in range(50):
        U = random_state(rng, G53)
        F = oracle.hllc(U, U, d, G53)
        Fp = oracle.flux(U, d, G53)
        assert np.allclose(F, Fp, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_stationary_contact_exact(d):
    # u_n = 0, equal pressure, density jump, arbitrary tangential velocity:
    # HLLC resolves it exactly: mass and energy flux 0, normal momentum flux P
    vt = np.array([0.3, -0.7, 0.2])
    vt[d] = 0.0
    WL = [1.0, *vt, 0.8]
    WR = [0.1, *(-vt), 0.8]
    F = oracle.hllc(oracle.cons(WL, G53), oracle.cons(WR, G53), d, G53)
    assert abs(F[0]) < 1e-15 and abs(F[4]) < 1e-15
    assert abs(F[1 + d] - 0.8) < 1e-15


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_supersonic_upwind_exact(d):
    rng = np.random.default_rng(20 + d)
    for sign in (+1, -1):
        WL = np.array([1.0, 0.1, -0.2, 0.3, 1.0])
        WR = np.array([0.5, 0.2, 0.1, -0.1, 0.6])
        WL[1 + d] = WR[1 + d] = sign * 6.0  # |u| > c_s + |du| for both
        UL, UR = oracle.cons(WL, G53), oracle.cons(WR, G53)
        F = oracle.hllc(UL, UR, d, G53)
        up = UL if sign > 0 else UR
        assert np.array_equal(F, oracle.flux(up, d, G53))


def test_hllc_mirror_antisymmetry():
    # reflecting x -> -x swaps L and R and flips v_x: F_mass, F_E change sign,
    # F_{mom x} is unchanged, F_{mom y,z} change sign
    rng = np.random.default_rng(3)
    for _ in range(50):
        UL, UR = random_state(rng, G53), random_state(rng, G53)
        M = np.array([1, -1, 1, 1, 1.0])
        F = oracle.hllc(UL, UR, 0, G53)
        Fm = oracle.hllc(UR * M, UL * M, 0, G53)
        assert np.allclose(Fm, -F * M, rtol=1e-13, atol=1e-14)


def test_vanleer_limiter_values():
    assert oracle.vanleer(1.0, 1.0) == 1.0
    assert oracle.vanleer(1.0, 3.0) == 1.5       # 2*3/4
    assert oracle.vanleer(-2.0, -2.0) == -2.0
    assert oracle.vanleer(1.0, -1.0) == 0.0       # extremum
    assert oracle.vanleer(0.0, 5.0) == 0.0


# ---- time step, Eq. CFL2 ---------------------------------------------------------

def test_dt_cfl2_hand_evaluated():
    U = ics.uniform_state(4, rho=2.0, v=(0.5, -1.0, 0.25), P=3.0, gamma=G53)
    cs = np.sqrt(G53 * 3.0 / 2.0)
    expect = 0.5 * 0.25 / (0.5 + 1.0 + 0.25 + 3 * cs)
    assert abs(oracle.dt_cfl2(U, G53, 0.5, 0.25) - expect) < 1e-15 * expect


# ---- whole step ------------------------------------------------------------------

def test_uniform_state_bit_identical():
    U = ics.uniform_state(8, gamma=G53)
    U1, _ = oracle.run_periodic(U, 1.0 / 8, G53, 0.5, 5)
    assert np.array_equal(U1, U)


def test_conservation_periodic():
    U = ics.sod_noise(16, seed=2, gamma=G53)
    s0 = oracle.conserved_sum(U, 1.0 / 16 ** 3)
    U1, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 4)
    s1 = oracle.conserved_sum(U1, 1.0 / 16 ** 3)
    scale = np.abs(U).sum(axis=(1, 2, 3)) / 16 ** 3
    assert np.all(np.abs(s1 - s0) <= 1e-14 * 4 * scale)


def test_mirror_symmetry_x():
    g = G53
    U = ics.sod_noise(16, seed=5, gamma=g)
    M = np.array([1, -1, 1, 1, 1.0])[:, None, None, None]
    Um = (U * M)[:, :, :, ::-1].copy()
    A, _ = oracle.run_periodic(U, 1.0 / 16, g, 0.5, 3)
    B, _ = oracle.run_periodic(Um, 1.0 / 16, g, 0.5, 3)
    Bm = (B * M)[:, :, :, ::-1]
    for v in range(5):
        assert rel_l1(Bm[v], A[v]) <= 1e-14 or np.abs(Bm[v] - A[v]).max() < 1e-14


def test_axis_permutation_symmetry():
    g = G53
    U = ics.sod_noise(16, seed=6, gamma=g)
    # x <-> y: transpose the last two axes and swap the x/y momenta
    P = U[[0, 2, 1, 3, 4]].transpose(0, 1, 3, 2).copy()
    A, _ = oracle.run_periodic(U, 1.0 / 16, g, 0.5, 3)
    B, _ = oracle.run_periodic(P, 1.0 / 16, g, 0.5, 3)
    Bp = B[[0, 2, 1, 3, 4]].transpose(0, 1, 3, 2)
    for v in range(5):
        assert rel_l1(Bp[v], A[v]) <= 1e-14 or np.abs(Bp[v] - A[v]).max() < 1e-14
    # x <-> z
    P = U[[0, 3, 2, 1, 4]].transpose(0, 3, 2, 1).copy()
    B, _ = oracle.run_periodic(P, 1.0 / 16, g, 0.5, 3)
    Bp = B[[0, 3, 2, 1, 4]].transpose(0, 3, 2, 1)
    for v in range(5):
        assert rel_l1(Bp[v], A[v]) <= 1e-14 or np.abs(Bp[v] - A[v]).max() < 1e-14


def run_to_time(U, dh, g, cfl, t_end):
    t = 0.0
    while t < t_end - 1e-15:
        dt = min(oracle.dt_cfl2(U, g, cfl, dh), t_end - t)
        U, nbad = oracle.step_periodic(U, dh, dt, g)
        assert nbad == 0
        t += dt
    return U


@pytest.mark.parametrize("g", [1.4, G53])
def test_sod_converges_to_exact(g):
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    t = 0.1
    errs = []
    for n in (64, 128, 256):
        U = ics.riemann_tube(n, L, R, axis=0, gamma=g)
        U = run_to_time(U, 1.0 / n, g, 0.5, t)
        # the solution is independent of y and z to the bit
        assert np.array_equal(U[:, :, :, :], np.broadcast_to(U[:, :1, :1, :], U.shape))
        x = ics.centres(n)
        sel = (x > 0.25) & (x < 0.75)  # away from the periodic wrap's second jump
        r, _, _ = oracle.exact_sample(L, R, g, (x[sel] - 0.5) / t)
        errs.append(np.abs(U[0, 0, 0, sel] - r).mean() * 0.5)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 4e-3
    order = np.log2(errs[0] / errs[2]) / 2
    assert order > 0.6, errs


def wave_error(n, direction, t_end, shape3d=False):
    g = G53
    k = np.asarray(direction, float)
    if shape3d:
        U = ics.advected_wave(n, direction, gamma=g)
    else:
        U = ics.advected_wave(n, direction, gamma=g, ny=4, nz=4)
    U = run_to_time(U, 1.0 / n, g, 0.5, t_end)
    if shape3d:
        x, y, z = ics.grid(n)
    else:
        x, y, z = ics.grid(n, 4, 4)
    # cell average of the exact solution rho(x - v t), v = k
    ph = 2 * np.pi * (k[0] * x + k[1] * y + k[2] * z - (k ** 2).sum() * t_end)
    fac = 1.0
    for kd in k:
        if kd != 0:
            a = np.pi * kd / n
            fac *= np.sin(a) / a
    exact = 1.0 + 0.2 * np.sin(ph) * fac
    return np.abs(U[0] - exact).mean()


def test_second_order_on_smooth_wave_x():
    e = [wave_error(n, (1, 0, 0), 0.25) for n in (32, 64, 128)]
    order = np.log2(e[0] / e[2]) / 2
    assert order >= 1.8, e


@pytest.mark.slow
def test_second_order_on_smooth_wave_diagonal():
    e = [wave_error(n, (1, 1, 1), 0.1, shape3d=True) for n in (16, 32)]
    order = np.log2(e[0] / e[1])
    assert order >= 1.6, e
