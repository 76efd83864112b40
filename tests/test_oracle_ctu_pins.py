"""Pins of the oracle's PPM reconstruction (Colella & Woodward 1984) and CTU
scheme (Colella 1990, the six-solve variant of Athena; section 2.2 lists both
and defers their details), against facts the mathematics fixes:

  * PPM face values: hand-evaluated cases of the interpolation and of both
    monotonicity constraints; exact face values of a quadratic's cell
    averages where the MC limiter picks the central slope; the constrained
    parabola is monotone inside every cell, for random data;
  * CTU: identical to the bit to MUSCL-Hancock on data varying along one axis
    (the transverse fluxes cancel exactly and the normal predictor is the
    Hancock step along that axis), with PLM and PPM;
  * every scheme (MUSCL-Hancock, VL, CTU) with PLM or PPM on a density
    profile carried diagonally at uniform velocity and pressure follows the
    textbook scalar advection scheme of the same construction, written out
    below for a scalar: this pins the transverse correction (its sign, its
    dt/2, and that it uses the cell's own first fluxes) and PPM inside whole
    steps;
  * Eq. CFL1 hand-evaluated;
  * the invariants (uniform state kept to the bit, conservation, mirror
    symmetry), Sod converging to the exact solution, and second order on a
    smooth diagonal wave at the CTU scheme's own Courant number 0.5 of
    Eq. CFL1.
"""
import numpy as np
import pytest

import oracle
from paper_1712_07070_b300 import ics
from test_oracle_pins import G53, rel_l1

LIMS = [(oracle.LIM_VANLEER, 1.5), (oracle.LIM_GMINMOD, 1.0), (oracle.LIM_GMINMOD, 2.0),
        (oracle.LIM_ALBADA, 1.5), (oracle.LIM_VL_GMINMOD, 1.3)]


# ---- PPM face values -------------------------------------------------------------

def test_ppm_hand_values():
    with oracle.scheme():  # van Leer-type slopes
        # smooth increasing data, no constraint active:
        # slopes vL(1,1) = 1, vL(1,2) = 4/3, vL(2,4) = 8/3;
        # W_L = 3/2 - (4/3 - 1)/6 = 13/9, W_R = 3 - (8/3 - 4/3)/6 = 25/9
        wl, wr = oracle.ppm_faces([0.0, 1.0, 2.0, 4.0, 8.0])
        assert abs(wl - 13 / 9) < 1e-15 and abs(wr - 25 / 9) < 1e-15
        # an extremum: both faces take the cell value
        assert oracle.ppm_faces([0.0, 1.0, 3.0, 1.0, 0.0]) == (3.0, 3.0)
        # the cell value near the right face: slopes vL(0.1,0.8) = vL(0.8,0.1) = 8/45,
        # vL(0.1,0) = 0; W_L = 1/2, W_R = 0.95 + (8/45)/6; d m > d^2 moves
        # W_L to 3 W_i - 2 W_R
        wr_e = 0.95 + 8 / 270
        wl, wr = oracle.ppm_faces([0.0, 0.1, 0.9, 1.0, 1.0])
        assert abs(wr - wr_e) < 1e-15 and abs(wl - (2.7 - 2 * wr_e)) < 1e-15
        # the mirror image moves W_R instead
        wl2, wr2 = oracle.ppm_faces([1.0, 1.0, 0.9, 0.1, 0.0])
        assert abs(wl2 - wr_e) < 1e-15 and abs(wr2 - (2.7 - 2 * wr_e)) < 1e-15


def test_ppm_exact_on_quadratic_averages():
    """Where the MC limiter (generalized minmod 2) selects the central slope,
    the face values of a quadratic's cell averages are the quadratic's point
    values at the faces."""
    q = lambda x: 0.3 + 2.0 * x + 0.4 * x * x  # increasing on [0, 2]
    Q = lambda x: 0.3 * x + x * x + 0.4 * x ** 3 / 3  # its antiderivative
    h = 0.05
    with oracle.scheme(oracle.LIM_GMINMOD, theta=2.0):
        for x0 in (0.2, 0.7, 1.3):
            avg = [(Q(x0 + (k + 0.5) * h) - Q(x0 + (k - 0.5) * h)) / h for k in range(-2, 3)]
            wl, wr = oracle.ppm_faces(avg)
            assert abs(wl - q(x0 - h / 2)) < 1e-13 and abs(wr - q(x0 + h / 2)) < 1e-13


@pytest.mark.parametrize("lim,theta", LIMS)
def test_ppm_parabola_monotone_in_cell(lim, theta):
    rng = np.random.default_rng(3)
    with oracle.scheme(lim, theta=theta):
        for _ in range(400):
            w = rng.normal(size=5) * rng.choice([1e-3, 1.0, 10.0])
            wl, wr = oracle.ppm_faces(w)
            c = w[2]
            a6 = 6.0 * (c - 0.5 * (wl + wr))
            # no interior extremum: |a6| <= |W_R - W_L| (flat allowed)
            assert abs(a6) <= abs(wr - wl) * (1 + 1e-12) + 1e-14, (w, wl, wr)


# ---- CTU reduces to MUSCL-Hancock in one dimension ---------------------------------

@pytest.mark.parametrize("ppm", [False, True])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ctu_equals_muscl_hancock_in_1d(ppm, axis):
    L, R = (1.0, 0.3, 1.0), (0.2, -0.1, 0.15)
    U = ics.riemann_tube(32, L, R, axis=axis, gamma=G53)
    rng = np.random.default_rng(axis)
    U = U * (1 + 0.02 * rng.normal(size=32)).reshape([-1 if 2 - axis == k else 1 for k in range(3)])
    dt = 0.3 / 32
    with oracle.scheme(ppm=ppm):
        a, _ = oracle.step_periodic(U, 1.0 / 32, dt, G53)
    with oracle.scheme(ctu=True, ppm=ppm):
        b, _ = oracle.step_periodic(U, 1.0 / 32, dt, G53)
    assert np.array_equal(a, b)


# ---- diagonal entropy waves: the scalar schemes --------------------------------------

def _lim(lim, theta, a, b):
    ab = a * b
    pos = ab > 0
    vl = np.where(pos, 2 * ab / np.where(pos, a + b, 1.0), 0.0)
    gm = np.where(pos, np.sign(a) * np.minimum(np.minimum(theta * np.abs(a), np.abs(a + b) / 2),
                                               theta * np.abs(b)), 0.0)
    if lim == oracle.LIM_VANLEER:
        return vl
    if lim == oracle.LIM_GMINMOD:
        return gm
    if lim == oracle.LIM_ALBADA:
        return np.where(pos, ab * (a + b) / np.where(pos, a * a + b * b, 1.0), 0.0)
    return np.where(np.abs(vl) < np.abs(gm), vl, gm)


def _sh(q, d, k):
    """q at the cell k cells further along d (arrays [z][y][x], periodic)."""
    return np.roll(q, -k, axis=2 - d)


def _faces(q, d, lim, theta, ppm):
    """Left and right face values of every cell along d."""
    s = lambda r: _lim(lim, theta, r - _sh(r, d, -1), _sh(r, d, 1) - r)
    if not ppm:
        sl = s(q)
        return q - sl / 2, q + sl / 2
    sl = s(q)
    right = (q + _sh(q, d, 1)) / 2 - (_sh(sl, d, 1) - sl) / 6  # W_{i+1/2}
    l, r = _sh(right, d, -1), right.copy()
    flat = (r - q) * (q - l) <= 0
    dd, m = r - l, 6 * (q - (l + r) / 2)
    up, dn = dd * m > dd * dd, dd * m < -dd * dd
    l2 = np.where(flat, q, np.where(up, 3 * q - 2 * r, l))
    r2 = np.where(flat, q, np.where(~up & dn, 3 * q - 2 * l, r))
    return l2, r2


def _scalar_step(q, nu, lim, theta, scheme, ppm):
    """One step of linear advection, velocity > 0 along every axis, Courant
    numbers nu[d]: upwind fluxes (times dt/dh) nu_d * (right face value)."""
    if scheme == "vl":
        qs = q - 0.5 * sum(nu[e] * (q - _sh(q, e, -1)) for e in range(3))
        F = [nu[d] * _faces(qs, d, lim, theta, ppm)[1] for d in range(3)]
    else:
        f = [_faces(q, d, lim, theta, ppm) for d in range(3)]
        if scheme == "mh":  # every face gets the Hancock increment of all directions
            inc = -0.5 * sum(nu[e] * (f[e][1] - f[e][0]) for e in range(3))
            F = [nu[d] * (f[d][1] + inc) for d in range(3)]
        else:  # ctu: normal predictor, first fluxes, transverse correction
            pred = [f[d][1] - 0.5 * nu[d] * (f[d][1] - f[d][0]) for d in range(3)]
            F1 = [nu[d] * pred[d] for d in range(3)]
            dF1 = [F1[d] - _sh(F1[d], d, -1) for d in range(3)]
            F = [nu[d] * (pred[d] - 0.5 * sum(dF1[e] for e in range(3) if e != d)) for d in range(3)]
    return q - sum(F[d] - _sh(F[d], d, -1) for d in range(3))


@pytest.mark.parametrize("rs", [oracle.RS_HLLC, oracle.RS_ROE, oracle.RS_EXACT])
@pytest.mark.parametrize("lim,theta", LIMS)
@pytest.mark.parametrize("scheme,ppm", [("mh", False), ("mh", True), ("vl", True), ("ctu", False), ("ctu", True)])
def test_diagonal_entropy_wave_is_scalar_advection(rs, lim, theta, scheme, ppm):
    n = 12
    vel = np.array([0.8, 0.6, 0.5])
    x, y, z = ics.grid(n)
    rho = 1.0 + 0.4 * np.sin(2 * np.pi * (x + 2 * y)) * np.cos(2 * np.pi * z) + \
        np.where((x - 0.5) ** 2 + (y - 0.4) ** 2 + (z - 0.6) ** 2 < 0.06, 0.6, 0.0)
    P = 1.0
    U = np.stack([rho, rho * vel[0], rho * vel[1], rho * vel[2],
                  P / (G53 - 1) + 0.5 * rho * (vel ** 2).sum()])
    dh = 1.0 / n
    dt = 0.45 * dh / vel[0]
    nu = vel * dt / dh
    ref = rho.copy()
    with oracle.scheme(lim, rs, theta, vl=scheme == "vl", ctu=scheme == "ctu", ppm=ppm):
        for _ in range(2):
            U, nbad = oracle.step_periodic(U, dh, dt, G53)
            assert nbad == 0
            ref = _scalar_step(ref, nu, lim, theta, scheme, ppm)
    assert np.abs(U[0] - ref).max() <= 2e-13
    for d in range(3):
        assert np.abs(U[1 + d] / U[0] - vel[d]).max() <= 2e-13
    assert np.abs((G53 - 1) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]) - P).max() <= 2e-13


# ---- Eq. CFL1 ---------------------------------------------------------------------

def test_dt_cfl1_hand_evaluated():
    # two cells: (rho, v, P) = (1, (0.3,-0.5,0.1), 0.6) and (2, (1,0,0), 1.2);
    # c_s = sqrt(gamma P / rho) = 1 in both (gamma = 5/3);
    # max(|v|) + c_s = 1.5 and 2.0 -> dt = 0.5 * 0.25 / 2
    U = np.zeros((5, 1, 1, 2))
    for i, (r, v, p) in enumerate([(1.0, (0.3, -0.5, 0.1), 0.6), (2.0, (1.0, 0.0, 0.0), 1.2)]):
        U[:, 0, 0, i] = oracle.cons([r, *v, p], G53)
    assert abs(oracle.max_speed1(U, G53) - 2.0) < 1e-15
    assert abs(oracle.dt_cfl1(U, G53, 0.5, 0.25) - 0.0625) < 1e-16
    with oracle.scheme(ctu=True):
        assert oracle.dt_cfl(U, G53, 0.5, 0.25) == oracle.dt_cfl1(U, G53, 0.5, 0.25)
    assert oracle.dt_cfl(U, G53, 0.5, 0.25) == oracle.dt_cfl2(U, G53, 0.5, 0.25)


# ---- invariants and convergence ----------------------------------------------------

SCHEMES = [dict(ctu=True), dict(ctu=True, ppm=True), dict(ppm=True), dict(vl=True, ppm=True),
           dict(ctu=True, riemann=oracle.RS_ROE, ppm=True),
           dict(ctu=True, limiter=oracle.LIM_GMINMOD, riemann=oracle.RS_HLLE)]


def run_to(U, dh, g, t_end, cfl=0.5):
    t = 0.0
    while t < t_end - 1e-15:
        dt = min(oracle.dt_cfl(U, g, cfl, dh), t_end - t)
        U, nbad = oracle.step_periodic(U, dh, dt, g)
        assert nbad == 0
        t += dt
    return U


@pytest.mark.parametrize("kw", SCHEMES)
def test_invariants(kw):
    with oracle.scheme(**kw):
        U = ics.uniform_state(8, gamma=G53)
        U1, _ = oracle.run_periodic(U, 1.0 / 8, G53, 0.5, 3)
        assert np.array_equal(U1, U)
        U = ics.sod_noise(16, seed=5, gamma=G53)
        s0 = oracle.conserved_sum(U, 1.0 / 16 ** 3)
        U1, _ = oracle.run_periodic(U, 1.0 / 16, G53, 0.5, 3)
        s1 = oracle.conserved_sum(U1, 1.0 / 16 ** 3)
        scale = np.abs(U).sum(axis=(1, 2, 3)) / 16 ** 3
        assert np.all(np.abs(s1 - s0) <= 1e-14 * 4 * scale)
        for ax in range(3):  # mirror along each axis
            M = np.ones(5)
            M[1 + ax] = -1
            M = M[:, None, None, None]
            flip = lambda a: np.flip(a, axis=3 - ax).copy()
            B, _ = oracle.run_periodic(flip(U * M), 1.0 / 16, G53, 0.5, 3)
            Bm = flip(B) * M
            for v in range(5):
                assert rel_l1(Bm[v], U1[v]) <= 1e-13 or np.abs(Bm[v] - U1[v]).max() < 1e-14


def sod_error(n, g=1.4, t=0.1):
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    U = run_to(ics.riemann_tube(n, L, R, axis=0, gamma=g), 1.0 / n, g, t)
    x = ics.centres(n)
    sel = (x > 0.25) & (x < 0.75)
    r, _, _ = oracle.exact_sample(L, R, g, (x[sel] - 0.5) / t)
    return np.abs(U[0, 0, 0, sel] - r).mean() * 0.5


@pytest.mark.parametrize("kw", SCHEMES)
def test_sod_converges(kw):
    with oracle.scheme(**kw):
        e = [sod_error(n) for n in (64, 128)]
    assert e[1] < e[0] and e[1] < 7e-3, e


def diagonal_wave_error(n, t_end=0.25):
    k = np.array([1.0, 1.0, 1.0])
    U = ics.advected_wave(n, tuple(k), gamma=G53, speed=0.5)
    U = run_to(U, 1.0 / n, G53, t_end)
    x, y, z = ics.grid(n)
    ph = 2 * np.pi * (x + y + z - 0.5 * 3 * t_end)
    fac = (np.sin(np.pi / n) / (np.pi / n)) ** 3
    exact = 1.0 + 0.2 * fac * np.sin(ph)
    return np.abs(U[0] - exact).mean()


@pytest.mark.parametrize("kw", [dict(ctu=True), dict(ctu=True, ppm=True), dict(ppm=True)])
def test_second_order_on_a_diagonal_wave(kw):
    with oracle.scheme(**kw):
        e = [diagonal_wave_error(n) for n in (16, 32, 48)]
    # (8 cells per wavelength are pre-asymptotic: the limiters clip the crests)
    assert e[1] < e[0] / 3
    assert np.log(e[1] / e[2]) / np.log(1.5) >= 1.75, e
