"""Pins of the oracle's self-gravity coupling on the AMR hierarchy (section
2.3 predictor-corrector inside the section 2.1 W-cycle) against facts fixed
independently of it:

  * G = 0 leaves every level bitwise the plain hierarchy's;
  * with nothing refined, the root evolves bitwise as the single-level
    coupled steps (predictor, FFT potential, corrector) with the same time
    steps -- so the hierarchy carries g^n from one step to the next;
  * mass is conserved to round-off across fix-up and regrid with gravity;
  * a stable Jeans wave (4 pi G rho0 = c_s^2 k^2 / 2) crossing refined
    bands still oscillates at omega^2 = c_s^2 k^2 - 4 pi G rho0 (a missing
    or wrong-signed coupling on any level moves its amplitude far off).
"""
import numpy as np
import pytest

import oracle
from oracle import poisson as PS
from oracle.amr import OracleHierarchy
from oracle.amr_gravity import GravityHierarchy
from paper_1712_07070_b300 import ics

G53 = 5.0 / 3.0


def blobs():
    return ics.blobs(32, seed=5, contrast=10.0, mach=1.0)


def test_zero_gravity_is_the_plain_hierarchy():
    U0 = blobs()
    # G = 0: the potential is zero whatever the SOR's iteration count
    H = GravityHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1, 1], G=0.0, iters=1)
    P = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1, 1])
    H.advance(0)
    P.advance(0)
    assert H.log == P.log
    for l in range(3):
        assert np.array_equal(H.lv[l].mask, P.lv[l].mask)
        p = H.present(l)
        assert np.array_equal(H.lv[l].U[:, p], P.lv[l].U[:, p]), l


def test_unrefined_root_is_the_uniform_coupled_step():
    U0 = blobs()
    G = 2.0
    H = GravityHierarchy(U0, lmax=1, gamma=G53, cfl=0.5, theta=1e9, nbuf=[1], G=G)
    assert H.lv[1].empty
    for _ in range(3):
        H.advance(0)
    dts = [dt for (l, dt) in H.log]
    dh = 1.0 / 32
    U = U0
    g = PS.accel_periodic(PS.poisson_root_periodic(U[0], dh, G), dh)
    for dt in dts:
        U, _, g, nbad = PS.step_gravity(U, g, dh, dt, G53, G)
        assert nbad == 0
    assert np.array_equal(U, H.lv[0].U)
    assert np.array_equal(g, H.lv[0].g)


def test_mass_conserved_across_fixup_and_regrid():
    U0 = blobs()
    # conservation holds whatever the SOR's iteration count
    H = GravityHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1, 1], G=2.0, iters=5)
    assert 0 < H.lv[1].mask.sum() < H.lv[1].mask.size and not H.lv[2].empty

    def mass():
        return sum(H.lv[l].U[0][H.leaf(l)].sum() * H.dh(l) ** 3 for l in range(3) if not H.lv[l].empty)

    m0 = mass()
    H.advance(0)
    assert abs(mass() - m0) <= 1e-14 * m0


def jeans_amr(t_end=0.08, theta=9.3e-6, sign=1.0, iters=8):
    """Jeans wave along x on a 64 x 8 x 8 root with refined bands where the
    normalised density gradient is largest (|sin kx| > 0.95); the density
    mode's amplitude (root cells, restricted under level 1) against
    A cos(omega t)."""
    rho0, P0, A = 1.0, 1.0, 1e-4
    cs2 = G53 * P0 / rho0
    k = 2 * np.pi
    G = 0.5 * cs2 * k * k / (4 * np.pi * rho0)
    n = 64
    x = (np.arange(n) + 0.5) / n
    U = np.zeros((5, 8, 8, n))
    rho = rho0 * (1 + A * np.cos(k * x))
    U[0] = rho
    U[4] = P0 * (rho / rho0) ** G53 / (G53 - 1)
    H = GravityHierarchy(U, lmax=1, gamma=G53, cfl=0.5, theta=theta, nbuf=[1], G=sign * G, iters=iters)
    refined = H.lv[1].mask.sum()
    while H.lv[0].t < t_end - 1e-14:
        H.advance(0, min(H.min_dt(0), t_end - H.lv[0].t))
    omega = np.sqrt(cs2 * k * k - 4 * np.pi * G * rho0)
    amp = 2 * np.mean((H.lv[0].U[0, 0, 0] - rho0) * np.cos(k * x)) / rho0  # root (restricted under level 1)
    return abs(amp - A * np.cos(omega * H.lv[0].t)) / A, refined, H.lv[1].mask.size


def test_jeans_wave_through_refined_bands():
    # measured 7.9e-5 with 8 SOR iterations per refined solve (5.4e-4 with
    # 20; with no gravity on the refined level 6.3e-2), with the opposite
    # sign 0.20
    err, refined, total = jeans_amr()
    assert 0 < refined < total  # coarse-fine interfaces crossed by the wave
    assert err < 5e-3, err
    err_wrong, _, _ = jeans_amr(sign=-1.0)  # the opposite gravity: another frequency
    assert err_wrong > 0.1, err_wrong


def test_refined_solve_takes_the_parent_potential_at_its_own_time():
    # parent times 1 and 2 with potentials 0 and phi: a refined solve at
    # t = 1.5 uses 0.5 phi (the midpoint), at 2 and beyond phi, at 1 zero
    U0 = blobs()
    H = GravityHierarchy(U0, lmax=1, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1], G=1.0, iters=5)
    assert not H.lv[1].empty
    c = H.lv[0]
    phi = c.phi.copy()
    c.t_prev, c.t = 1.0, 2.0
    c.phi_prev = np.zeros_like(phi)
    assert H.parent_weight(1, 1.5) == 0.5
    assert H.parent_weight(1, 1.0) == 0.0
    assert H.parent_weight(1, 2.0) == H.parent_weight(1, 2.0 + 1e-15) == 1.0
    rho = H.lv[1].U[0]
    got_phi, got_g = H.solve_level(1, 1.5, rho)
    c.t_prev = c.t  # a single parent time: its newest potential
    c.phi = 0.5 * phi
    want_phi, want_g = H.solve_level(1, 1.5, rho)
    assert np.array_equal(got_phi, want_phi) and np.array_equal(got_g, want_g)
