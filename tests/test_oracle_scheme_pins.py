"""Pins of the oracle's other slope limiters and of the HLLE solver (section
2.2 lists them; definitions from Toro 2009 and Einfeldt 1991), against facts
the mathematics fixes -- never against the oracle itself:

  * limiters: hand-evaluated values, zero at extrema, exact on linear data,
    symmetry and oddness, Sweby's TVD region 0 <= phi(r) <= min(2r, 2), the
    generalized minmod at theta = 1 being the classical minmod, and the
    hybrid equal to the classical minmod at theta = 1 and to the van
    Leer-type limiter at theta = 2 (the latter never exceeds the MC bound);
  * HLLE: consistency F(U,U) = F(U), exact upwinding of supersonic states,
    mirror antisymmetry, and the diffusion of a stationary contact that HLLC
    resolves exactly;
  * Roe: consistency, upwinding, mirror antisymmetry, exact resolution of a
    stationary contact with shear and of a stationary Rankine-Hugoniot shock
    (Roe's property: any slip in the averages or eigenvectors breaks it),
    and convergence on a sonic rarefaction (which needs the entropy fix);
  * exact solver: the Godunov flux of the Sod problem from Toro's published
    star state (Table 4.2), consistency, upwinding, contact, mirror;
  * the VL half step (Riemann fluxes of the cell averages): the scheme
    invariants, Sod convergence, second order on a smooth wave (first order
    if the half step were lost), and a result that differs from
    MUSCL-Hancock's;
  * every scheme: uniform states unchanged to the bit, conservation to
    round-off, mirror symmetry, Sod converging to the exact solution, second
    order on a smooth wave, and the diffusion ordering the definitions imply
    (minmod > generalized minmod 1.5 > MC; HLLE > HLLC on a contact).
"""
import numpy as np
import pytest

import oracle
from paper_1712_07070_b300 import ics
from test_oracle_pins import G53, random_state, rel_l1, run_to_time, wave_error

LIMS = [oracle.LIM_VANLEER, oracle.LIM_GMINMOD, oracle.LIM_ALBADA, oracle.LIM_VL_GMINMOD]


def lim_fn(lim, theta=1.5):
    return {
        oracle.LIM_VANLEER: lambda a, b: oracle.vanleer(a, b),
        oracle.LIM_GMINMOD: lambda a, b: oracle.gminmod(a, b, theta),
        oracle.LIM_ALBADA: lambda a, b: oracle.albada(a, b),
        oracle.LIM_VL_GMINMOD: lambda a, b: oracle.vl_gminmod(a, b, theta),
    }[lim]


# ---- limiters ------------------------------------------------------------------

def test_limiter_hand_values():
    # a = 1, b = 3: vL 2*3/4, minmod family min(theta, 2, 3theta), albada 3*4/10
    assert oracle.gminmod(1.0, 3.0, 1.0) == 1.0
    assert oracle.gminmod(1.0, 3.0, 1.5) == 1.5
    assert oracle.gminmod(1.0, 3.0, 2.0) == 2.0
    assert oracle.albada(1.0, 3.0) == pytest.approx(1.2, rel=1e-15)
    assert oracle.vl_gminmod(1.0, 3.0, 1.0) == 1.0   # min(1.5, 1)
    assert oracle.vl_gminmod(1.0, 3.0, 1.5) == 1.5   # min(1.5, 1.5)
    # a = 4, b = 1: the central difference 2.5 binds MC, theta|b| binds 1.5
    assert oracle.gminmod(4.0, 1.0, 2.0) == 2.0
    assert oracle.gminmod(4.0, 1.0, 1.5) == 1.5
    # a = -1, b = -10
    assert oracle.gminmod(-1.0, -10.0, 1.5) == -1.5
    assert oracle.albada(-1.0, -10.0) == pytest.approx(-110.0 / 101.0, rel=1e-15)
    assert oracle.vl_gminmod(-1.0, -10.0, 2.0) == pytest.approx(-20.0 / 11.0, rel=1e-15)


@pytest.mark.parametrize("lim", LIMS)
def test_limiter_extrema_linear_symmetry(lim):
    f = lim_fn(lim)
    for a, b in [(1.0, -1.0), (0.0, 5.0), (5.0, 0.0), (-1.0, 2.0), (0.0, 0.0)]:
        assert f(a, b) == 0.0
    for a in (1.0, -2.0, 0.3, 7e-9):
        assert f(a, a) == pytest.approx(a, rel=1e-15)
    rng = np.random.default_rng(4)
    for _ in range(200):
        a, b = rng.normal(size=2) * 10.0 ** rng.uniform(-3, 3, 2)
        assert f(a, b) == f(b, a)
        assert f(-a, -b) == -f(a, b)


@pytest.mark.parametrize("lim", LIMS)
@pytest.mark.parametrize("theta", [1.0, 1.5, 2.0])
def test_limiter_in_tvd_region(lim, theta):
    f = lim_fn(lim, theta)
    for r in np.concatenate([np.linspace(1e-3, 5.0, 500), [10.0, 50.0, 1e3]]):
        phi = f(1.0, r)
        assert 0.0 <= phi <= min(2.0 * r, 2.0) * (1 + 1e-15), (r, phi)


def test_minmod_and_hybrid_identities():
    rng = np.random.default_rng(5)
    for _ in range(500):
        a, b = rng.normal(size=2) * 10.0 ** rng.uniform(-3, 3, 2)
        mm = np.sign(a) * min(abs(a), abs(b)) if a * b > 0 else 0.0
        assert oracle.gminmod(a, b, 1.0) == mm
        assert oracle.vl_gminmod(a, b, 1.0) == mm
        assert oracle.vl_gminmod(a, b, 2.0) == oracle.vanleer(a, b)


def test_hybrid_steps_equal_minmod_and_vanleer():
    # the identities above, through whole steps of the scheme (bitwise)
    U = ics.sod_noise(16, seed=9, gamma=G53)
    with oracle.scheme(oracle.LIM_VL_GMINMOD, theta=2.0):
        A, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 2)
    with oracle.scheme(oracle.LIM_VANLEER):
        B, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 2)
    assert np.array_equal(A, B)
    with oracle.scheme(oracle.LIM_VL_GMINMOD, theta=1.0):
        A, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 2)
    with oracle.scheme(oracle.LIM_GMINMOD, theta=1.0):
        B, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 2)
    assert np.array_equal(A, B)


# ---- HLLE ------------------------------------------------------------------------

@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlle_consistency_and_upwinding(d):
    rng = np.random.default_rng(30 + d)
    for _ in range(50):
        U = random_state(rng, G53)
        assert np.allclose(oracle.hlle(U, U, d, G53), oracle.flux(U, d, G53), rtol=1e-14, atol=1e-14)
    for sign in (+1, -1):
        WL = np.array([1.0, 0.1, -0.2, 0.3, 1.0])
        WR = np.array([0.5, 0.2, 0.1, -0.1, 0.6])
        WL[1 + d] = WR[1 + d] = sign * 6.0
        UL, UR = oracle.cons(WL, G53), oracle.cons(WR, G53)
        up = UL if sign > 0 else UR
        assert np.array_equal(oracle.hlle(UL, UR, d, G53), oracle.flux(up, d, G53))


def test_hlle_mirror_antisymmetry():
    rng = np.random.default_rng(6)
    M = np.array([1, -1, 1, 1, 1.0])
    for _ in range(50):
        UL, UR = random_state(rng, G53), random_state(rng, G53)
        F = oracle.hlle(UL, UR, 0, G53)
        Fm = oracle.hlle(UR * M, UL * M, 0, G53)
        assert np.allclose(Fm, -F * M, rtol=1e-13, atol=1e-14)


def test_hlle_diffuses_a_stationary_contact():
    # HLLC resolves it exactly; HLLE's single intermediate state smears it.
    # At rest with equal pressure F_L = F_R = (0, P, 0, 0, 0) and
    # E_L = E_R, so the HLLE formula gives mass flux
    # -S_L S_R (rho_R - rho_L)/(S_R - S_L) > 0 (down the density jump, since
    # S_L < 0 < S_R), normal-momentum flux P exactly and no energy flux.
    WL, WR = [1.0, 0.0, 0.0, 0.0, 0.8], [0.1, 0.0, 0.0, 0.0, 0.8]
    UL, UR = oracle.cons(WL, G53), oracle.cons(WR, G53)
    Fc = oracle.hllc(UL, UR, 0, G53)
    Fe = oracle.hlle(UL, UR, 0, G53)
    assert Fc[0] == 0.0
    assert Fe[0] > 1e-3
    assert Fe[1] == pytest.approx(0.8, rel=1e-15) and Fe[4] == 0.0


# ---- Roe and the exact solver --------------------------------------------------

SOLVERS = {"roe": oracle.roe, "exact": oracle.exact_flux}


@pytest.mark.parametrize("name", ["roe", "exact"])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_solver_consistency_upwinding_contact(name, d):
    f = SOLVERS[name]
    rng = np.random.default_rng(50 + d)
    for _ in range(30):
        U = random_state(rng, G53)
        assert np.allclose(f(U, U, d, G53), oracle.flux(U, d, G53), rtol=1e-13, atol=1e-13)
    for sign in (+1, -1):
        WL = np.array([1.0, 0.1, -0.2, 0.3, 1.0])
        WR = np.array([0.5, 0.2, 0.1, -0.1, 0.6])
        WL[1 + d] = WR[1 + d] = sign * 6.0
        UL, UR = oracle.cons(WL, G53), oracle.cons(WR, G53)
        up = UL if sign > 0 else UR
        assert np.allclose(f(UL, UR, d, G53), oracle.flux(up, d, G53), rtol=1e-13, atol=1e-13)
    vt = np.array([0.3, -0.7, 0.2])
    vt[d] = 0.0
    F = f(oracle.cons([1.0, *vt, 0.8], G53), oracle.cons([0.1, *(-vt), 0.8], G53), d, G53)
    assert abs(F[0]) < 1e-15 and abs(F[4]) < 1e-15 and abs(F[1 + d] - 0.8) < 1e-15


@pytest.mark.parametrize("name", ["roe", "exact"])
def test_solver_mirror_antisymmetry(name):
    f = SOLVERS[name]
    rng = np.random.default_rng(7)
    M = np.array([1, -1, 1, 1, 1.0])
    for _ in range(30):
        UL, UR = random_state(rng, G53), random_state(rng, G53)
        assert np.allclose(f(UR * M, UL * M, 0, G53), -f(UL, UR, 0, G53) * M, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("g", [1.4, G53])
def test_roe_resolves_a_stationary_shock(g):
    # Rankine-Hugoniot, upstream Mach 2 moving right into a shock at rest
    M1, r1, p1 = 2.0, 1.0, 1.0
    u1 = M1 * np.sqrt(g * p1 / r1)
    r2 = r1 * (g + 1) * M1 ** 2 / ((g - 1) * M1 ** 2 + 2)
    p2 = p1 * (1 + 2 * g / (g + 1) * (M1 ** 2 - 1))
    u2 = u1 * r1 / r2
    UL, UR = oracle.cons([r1, u1, 0.3, -0.1, p1], g), oracle.cons([r2, u2, 0.3, -0.1, p2], g)
    FL = oracle.flux(UL, 0, g)
    assert np.allclose(oracle.flux(UR, 0, g), FL, rtol=1e-13)  # the jump conditions hold
    assert np.allclose(oracle.roe(UL, UR, 0, g), FL, rtol=1e-12, atol=1e-13)


def test_exact_flux_of_sod_from_published_star_state():
    # Toro (2009) Table 4.2, test 1: p* = 0.30313, u* = 0.92745, rho*_L = 0.42632;
    # x/t = 0 lies between the left rarefaction's tail and the contact
    g = 1.4
    F = oracle.exact_flux(oracle.cons([1.0, 0, 0, 0, 1.0], g), oracle.cons([0.125, 0, 0, 0, 0.1], g), 0, g)
    r, u, p = 0.42632, 0.92745, 0.30313
    E = p / (g - 1) + 0.5 * r * u * u
    assert np.allclose(F, [r * u, r * u * u + p, 0, 0, (E + p) * u], rtol=3e-5, atol=0)


def test_roe_entropy_fix_sonic_rarefaction():
    # Toro's test with a sonic point in the left rarefaction (rho, u, p) =
    # (1, 0.75, 1) | (0.125, 0, 0.1): without an entropy fix Roe's solver
    # keeps an expansion shock at x/t ~ 0 and the error stops converging
    L, R, g, t = (1.0, 0.75, 1.0), (0.125, 0.0, 0.1), 1.4, 0.1
    errs = []
    with oracle.scheme(oracle.LIM_VANLEER, oracle.RS_ROE):
        for n in (64, 128, 256):
            U = ics.riemann_tube(n, L, R, axis=0, gamma=g)
            U = run_to_time(U, 1.0 / n, g, 0.5, t)
            x = ics.centres(n)
            sel = (x > 0.3) & (x < 0.7)
            r, _, _ = oracle.exact_sample(L, R, g, (x[sel] - 0.5) / t)
            errs.append(np.abs(U[0, 0, 0, sel] - r).mean())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 4e-3, errs
    assert np.log2(errs[0] / errs[2]) / 2 > 0.6, errs


# ---- whole steps of every scheme ----------------------------------------------------

SCHEMES = [(oracle.LIM_VANLEER, oracle.RS_HLLE, 1.5, False), (oracle.LIM_GMINMOD, oracle.RS_HLLC, 1.5, False),
           (oracle.LIM_GMINMOD, oracle.RS_HLLE, 2.0, False), (oracle.LIM_ALBADA, oracle.RS_HLLC, 1.5, False),
           (oracle.LIM_VL_GMINMOD, oracle.RS_HLLC, 1.5, False), (oracle.LIM_VANLEER, oracle.RS_ROE, 1.5, False),
           (oracle.LIM_GMINMOD, oracle.RS_EXACT, 1.5, False),
           # the VL half step (Riemann fluxes of the cell averages)
           (oracle.LIM_VANLEER, oracle.RS_HLLC, 1.5, True), (oracle.LIM_GMINMOD, oracle.RS_HLLE, 1.5, True)]


@pytest.mark.parametrize("lim,rs,theta,vl", SCHEMES)
def test_scheme_invariants(lim, rs, theta, vl):
    with oracle.scheme(lim, rs, theta, vl):
        U = ics.uniform_state(8, gamma=G53)
        U1, _ = oracle.run_periodic(U, 1.0 / 8, G53, 0.5, 3)
        assert np.array_equal(U1, U)
        U = ics.sod_noise(16, seed=2, gamma=G53)
        s0 = oracle.conserved_sum(U, 1.0 / 16 ** 3)
        U1, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 3)
        s1 = oracle.conserved_sum(U1, 1.0 / 16 ** 3)
        scale = np.abs(U).sum(axis=(1, 2, 3)) / 16 ** 3
        assert np.all(np.abs(s1 - s0) <= 1e-14 * 4 * scale)
        M = np.array([1, -1, 1, 1, 1.0])[:, None, None, None]
        Um = (U * M)[:, :, :, ::-1].copy()
        B, _ = oracle.run_periodic(Um, 1.0 / 16, G53, 0.5, 3)
        Bm = (B * M)[:, :, :, ::-1]
        for v in range(5):
            assert rel_l1(Bm[v], U1[v]) <= 1e-14 or np.abs(Bm[v] - U1[v]).max() < 1e-14


def sod_error(n, g=G53, t=0.1):
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    U = ics.riemann_tube(n, L, R, axis=0, gamma=g)
    U = run_to_time(U, 1.0 / n, g, 0.5, t)
    x = ics.centres(n)
    sel = (x > 0.25) & (x < 0.75)
    r, _, _ = oracle.exact_sample(L, R, g, (x[sel] - 0.5) / t)
    return np.abs(U[0, 0, 0, sel] - r).mean() * 0.5


@pytest.mark.parametrize("lim,rs,theta,vl", SCHEMES)
def test_scheme_sod_and_smooth_wave(lim, rs, theta, vl):
    with oracle.scheme(lim, rs, theta, vl):
        e = [sod_error(n) for n in (64, 128)]
        assert e[0] > e[1] and e[1] < 7e-3, e
        w = [wave_error(n, (1, 0, 0), 0.25) for n in (32, 64, 128)]
    order = np.log2(w[0] / w[2]) / 2
    assert order >= 1.75, w


def test_diffusion_ordering():
    errs = {}
    for key, args in {"minmod": (oracle.LIM_GMINMOD, oracle.RS_HLLC, 1.0),
                      "gmm15": (oracle.LIM_GMINMOD, oracle.RS_HLLC, 1.5),
                      "mc": (oracle.LIM_GMINMOD, oracle.RS_HLLC, 2.0),
                      "vl_hllc": (oracle.LIM_VANLEER, oracle.RS_HLLC, 1.5),
                      "vl_hlle": (oracle.LIM_VANLEER, oracle.RS_HLLE, 1.5)}.items():
        with oracle.scheme(*args):
            errs[key] = sod_error(128)
    assert errs["minmod"] > errs["gmm15"] > errs["mc"], errs
    assert errs["vl_hlle"] > errs["vl_hllc"], errs


def test_vl_differs_from_muscl_hancock():
    U = ics.sod_noise(16, seed=4, gamma=G53)
    with oracle.scheme(vl=True):
        A, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 2)
    B, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 2)
    d = rel_l1(A[0], B[0])
    assert 1e-6 < d < 1e-1, d


def _scalar_limiter(lim, theta, a, b):
    """The limited slope of a scalar (the section 2.2 limiters, written out)."""
    ab = a * b
    pos = ab > 0
    vl = np.where(pos, 2 * ab / np.where(pos, a + b, 1.0), 0.0)
    gm = np.where(pos, np.sign(a) * np.minimum(np.minimum(theta * np.abs(a), np.abs(a + b) / 2), theta * np.abs(b)), 0.0)
    if lim == oracle.LIM_VANLEER:
        return vl
    if lim == oracle.LIM_GMINMOD:
        return gm
    if lim == oracle.LIM_ALBADA:
        return np.where(pos, ab * (a + b) / np.where(pos, a * a + b * b, 1.0), 0.0)
    return np.where(np.abs(vl) < np.abs(gm), vl, gm)


def _scalar_step(rho, nu, lim, theta, vl):
    """One step of linear advection (speed > 0, Courant number nu) by the
    MUSCL-Hancock scheme (face value rho_i + (1 - nu) s_i / 2) or the VL
    scheme (upwind half step rho*, face value rho*_i + s*_i / 2), s the
    limited slope, conservative upwind update of rho^n."""
    m = lambda q: np.roll(q, 1)   # q_{i-1}
    p = lambda q: np.roll(q, -1)  # q_{i+1}
    if vl:
        r = rho - 0.5 * nu * (rho - m(rho))
        face = r + 0.5 * _scalar_limiter(lim, theta, r - m(r), p(r) - r)
    else:
        face = rho + 0.5 * (1 - nu) * _scalar_limiter(lim, theta, rho - m(rho), p(rho) - rho)
    return rho - nu * (face - m(face))


@pytest.mark.parametrize("rs", [oracle.RS_HLLC, oracle.RS_ROE, oracle.RS_EXACT])
@pytest.mark.parametrize("lim,theta", [(oracle.LIM_VANLEER, 1.5), (oracle.LIM_GMINMOD, 1.0),
                                       (oracle.LIM_GMINMOD, 2.0), (oracle.LIM_ALBADA, 1.5),
                                       (oracle.LIM_VL_GMINMOD, 1.3)])
@pytest.mark.parametrize("vl", [False, True])
def test_entropy_wave_reduces_to_scalar_advection(rs, lim, theta, vl):
    """A density profile carried at uniform velocity and pressure: HLLC, Roe
    and the exact solver resolve its contacts exactly, velocity and pressure
    stay uniform, and the density follows the textbook scalar advection
    scheme of the same reconstruction (MUSCL-Hancock or VL) exactly.  Catches
    a dropped half step, a wrong Courant factor or a shifted slope index."""
    n, u, nu = 32, 0.8, 0.45
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.5 * np.sin(2 * np.pi * x) + np.where((x > 0.3) & (x < 0.55), 0.7, 0.0)
    P = 1.0
    U = np.zeros((5, 2, 2, n))
    U[0] = rho
    U[1] = rho * u
    U[4] = P / (G53 - 1) + 0.5 * rho * u * u
    dh = 1.0 / n
    dt = nu * dh / u
    ref = rho.copy()
    with oracle.scheme(lim, rs, theta, vl):
        for _ in range(3):
            U, nbad = oracle.step_periodic(U, dh, dt, G53)
            assert nbad == 0
            ref = _scalar_step(ref, nu, lim, theta, vl)
    assert np.abs(U[0] - ref).max() <= 1e-13
    assert np.abs(U[1] / U[0] - u).max() <= 1e-13
    assert np.abs((G53 - 1) * (U[4] - 0.5 * U[1] ** 2 / U[0]) - P).max() <= 1e-13
    assert np.abs(U[2:4]).max() <= 1e-14
