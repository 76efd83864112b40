"""Pins of the gravity oracle (oracle/poisson.py; section 2.3 and Appendix A):

  * root FFT solution: its 7-point discrete Laplacian is 4 pi G (rho - <rho>)
    to round-off, and a single Fourier mode gives the closed form
    4 pi G A dh^2 / lambda_k;
  * quadratic interpolation reproduces a tensor-product quadratic exactly;
  * SOR: one iteration on a 4^3 grid written out cell by cell in red-black
    order, and convergence to the direct sparse solution of the discrete
    Dirichlet problem on an 18^3 grid;
  * central differences: the two-point form exact on quadratics, the
    four-point form on quartics.
"""
import numpy as np
import pytest

from oracle import poisson as PS


def test_root_solution_satisfies_the_discrete_equation():
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.3 * rng.random((16, 24, 32))
    dh, G = 1.0 / 32, 0.7
    phi = PS.poisson_root_periodic(rho, dh, G)
    lap = PS.laplacian_periodic(phi, dh)
    rhs = 4 * np.pi * G * (rho - rho.mean())
    assert np.abs(lap - rhs).max() <= 1e-10 * np.abs(rhs).max()
    assert abs(phi.mean()) <= 1e-12 * np.abs(phi).max()


def test_root_single_mode_closed_form():
    n, k, A, G = 32, 3, 0.2, 1.0
    dh = 1.0 / n
    x = np.arange(n)
    rho = 1.0 + A * np.sin(2 * np.pi * k * x / n)[None, None, :] * np.ones((8, 16, 1))
    phi = PS.poisson_root_periodic(rho, dh, G)
    lam = -2.0 * (1 - np.cos(2 * np.pi * k / n))
    expect = 4 * np.pi * G * A * dh * dh / lam * np.sin(2 * np.pi * k * x / n)
    assert np.abs(phi - expect[None, None, :]).max() <= 1e-13 * np.abs(expect).max()


def test_quadratic_interpolation_exact_on_quadratics():
    nc = 16
    q = lambda x, y, z: (0.3 + 1.1 * x - 0.7 * x * x) * (1.0 + 0.4 * y + 0.2 * y * y) + 0.5 * z * z - z
    c = np.arange(nc) + 0.5  # coarse centres (coarse units)
    phi_c = q(c[None, None, :], c[None, :, None], c[:, None, None])
    f = np.arange(6, 20)  # fine cells away from the periodic wrap
    out = PS.interp_quadratic(phi_c, f, f, f)
    xf = (f + 0.5) / 2.0  # fine centres in coarse units
    ref = q(xf[None, None, :], xf[None, :, None], xf[:, None, None])
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


def test_sor_one_iteration_by_hand():
    rng = np.random.default_rng(2)
    phi0 = rng.random((4, 4, 4))
    rho = rng.random((4, 4, 4))
    dh, G, om = 0.1, 1.3, 1.7
    out = PS.sor(phi0, rho, dh, G, om, 1)
    p = phi0.copy()
    for colour in (0, 1):
        for k in range(1, 3):
            for j in range(1, 3):
                for i in range(1, 3):
                    if (i + j + k) % 2 != colour:
                        continue
                    nb = p[k - 1, j, i] + p[k + 1, j, i] + p[k, j - 1, i] + p[k, j + 1, i] + p[k, j, i - 1] + p[k, j, i + 1]
                    p[k, j, i] += om * (nb - 6 * p[k, j, i] - dh * dh * 4 * np.pi * G * rho[k, j, i]) / 6
    assert np.allclose(out, p, rtol=0, atol=1e-15)


def test_sor_converges_to_the_direct_solution():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    n, m = 18, 16
    rng = np.random.default_rng(3)
    phi0 = rng.random((n, n, n))
    rho = rng.random((n, n, n))
    dh, G = 0.05, 1.0
    phi = PS.sor(phi0, rho, dh, G, 1.75, 300)
    # direct: interior unknowns, boundary values moved to the right-hand side
    idx = -np.ones((n, n, n), int)
    idx[1:-1, 1:-1, 1:-1] = np.arange(m ** 3).reshape(m, m, m)
    rows, cols, vals = [], [], []
    b = dh * dh * 4 * np.pi * G * rho[1:-1, 1:-1, 1:-1].ravel().copy()
    for k in range(1, n - 1):
        for j in range(1, n - 1):
            for i in range(1, n - 1):
                r = idx[k, j, i]
                rows.append(r); cols.append(r); vals.append(-6.0)
                for dk, dj, di in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    c = idx[k + dk, j + dj, i + di]
                    if c >= 0:
                        rows.append(r); cols.append(c); vals.append(1.0)
                    else:
                        b[r] -= phi0[k + dk, j + dj, i + di]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m ** 3, m ** 3))
    x = spl.spsolve(A, b).reshape(m, m, m)
    assert np.abs(phi[1:-1, 1:-1, 1:-1] - x).max() <= 1e-11 * np.abs(x).max()
    assert np.array_equal(phi[0], phi0[0]) and np.array_equal(phi[:, -1], phi0[:, -1])


@pytest.mark.parametrize("order,deg", [(2, 2), (4, 4)])
def test_central_differences_exact_on_polynomials(order, deg):
    n, dh = 12, 0.1
    x = np.arange(n) * dh
    coef = np.random.default_rng(4).random(deg + 1)
    poly = lambda t: sum(c * t ** p for p, c in enumerate(coef))
    dpoly = lambda t: sum(p * c * t ** (p - 1) for p, c in enumerate(coef) if p)
    phi = poly(x)[None, None, :] + 2 * poly(x)[None, :, None] - poly(x)[:, None, None]
    g = PS.accel(phi, dh, order)
    h = order // 2
    xi = x[h:n - h]
    assert np.allclose(g[0], -dpoly(xi)[None, None, :], rtol=1e-10, atol=1e-10)
    assert np.allclose(g[1], -2 * dpoly(xi)[None, :, None], rtol=1e-10, atol=1e-10)
    assert np.allclose(g[2], dpoly(xi)[:, None, None], rtol=1e-10, atol=1e-10)


# ---- the gravity coupling (predictor-corrector) -------------------------------------

G53 = 5.0 / 3.0


def test_predictor_with_zero_field_is_the_plain_step():
    import oracle
    from paper_1712_07070_b300 import ics
    U = ics.sod_noise(16, seed=6, gamma=G53)
    dt = oracle.dt_cfl2(U, G53, 0.5, 1 / 16)
    a, _ = oracle.step_periodic(U, 1 / 16, dt, G53)
    b, _ = oracle.step_gravity_predictor(U, np.zeros((3,) + U.shape[1:]), 1 / 16, dt, G53)
    assert np.array_equal(a, b)


def test_uniform_state_in_a_constant_field_falls_freely():
    """The predictor leaves a uniform state unchanged (equal fluxes on all
    faces); the corrector gives it the momentum rho g dt and exactly the
    kinetic energy of the new velocity, the pressure unchanged."""
    import oracle
    rho, v, P = 1.3, np.array([0.2, -0.1, 0.05]), 0.7
    U = np.zeros((5, 4, 4, 4))
    U[0] = rho
    U[1:4] = (rho * v)[:, None, None, None]
    U[4] = P / (G53 - 1) + 0.5 * rho * (v @ v)
    g = np.broadcast_to(np.array([0.3, 0.5, -0.2])[:, None, None, None], (3, 4, 4, 4)).copy()
    dt = 0.01
    Us, _ = oracle.step_gravity_predictor(U, g, 1 / 4, dt, G53)
    assert np.array_equal(Us, U)
    out = PS.gravity_correct(U, g, Us, g, dt)
    v1 = v + dt * g[:, 0, 0, 0]
    assert np.allclose(out[1:4], (rho * v1)[:, None, None, None], rtol=1e-15, atol=0)
    assert np.allclose(out[4], P / (G53 - 1) + 0.5 * rho * (v1 @ v1), rtol=1e-15, atol=0)


def jeans_amplitude_error(n, t_end=0.3):
    """A small sinusoidal perturbation of a self-gravitating uniform medium
    (stable: 4 pi G rho0 = c_s^2 k^2 / 2) oscillates with
    omega^2 = c_s^2 k^2 - 4 pi G rho0; the error of the density mode's
    amplitude against A cos(omega t)."""
    import oracle
    rho0, P0, A = 1.0, 1.0, 1e-4
    cs2 = G53 * P0 / rho0
    k = 2 * np.pi
    G = 0.5 * cs2 * k * k / (4 * np.pi * rho0)
    x = (np.arange(n) + 0.5) / n
    U = np.zeros((5, 2, 2, n))
    rho = rho0 * (1 + A * np.cos(k * x))
    U[0] = rho
    U[4] = P0 * (rho / rho0) ** G53 / (G53 - 1)  # adiabatic perturbation
    dh = 1.0 / n
    g = PS.accel_periodic(PS.poisson_root_periodic(U[0], dh, G), dh)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(oracle.dt_cfl2(U, G53, 0.5, dh), t_end - t)
        U, _, g, nbad = PS.step_gravity(U, g, dh, dt, G53, G)
        assert nbad == 0
        t += dt
    omega = np.sqrt(cs2 * k * k - 4 * np.pi * G * rho0)
    amp = 2 * np.mean((U[0, 0, 0] - rho0) * np.cos(k * x)) / rho0
    return abs(amp - A * np.cos(omega * t_end)) / A


def test_jeans_oscillation_converges():
    e = [jeans_amplitude_error(n) for n in (16, 32, 64)]
    assert e[1] < e[0] and np.log2(e[1] / e[2]) >= 1.7, e
    assert e[2] < 2.5e-3, e  # measured 2.0e-3


def test_acceleration_time_step_closed_form():
    """Eq. (acc) on the two-point acceleration of phi = A cos(k y): the
    discrete g_y = A sin(k dh) sin(k y_j) / dh peaks at the cell centres
    nearest the quarter period, |sin| = cos(pi / n) for n a multiple of 4;
    the other components vanish."""
    n, A, c = 32, -0.7, 0.4
    dh = 1.0 / n
    y = (np.arange(n) + 0.5) * dh
    phi = np.broadcast_to((A * np.cos(2 * np.pi * y))[None, :, None], (8, n, 16)).copy()
    g = PS.accel_periodic(phi, dh, 2)
    gmax = abs(A) * np.sin(2 * np.pi * dh) * np.cos(np.pi / n) / dh
    assert np.abs(g[0]).max() == 0 and np.abs(g[2]).max() == 0
    assert PS.dt_acc(g, dh, c) == pytest.approx(c * np.sqrt(dh / gmax), rel=1e-14)


def test_isolated_fft_is_the_pairwise_sum():
    """The zero-padded FFT convolution equals the direct sum over all pairs
    of cell point masses (no self term), inside the box and on the two
    layers outside it that the four-point accelerations read."""
    rng = np.random.default_rng(5)
    rho = rng.random((5, 6, 7))
    dh, G = 0.3, 1.3
    direct = PS.pairwise_potential(rho, dh, G)
    fft = PS.poisson_root_isolated(rho, dh, G)
    assert np.abs(fft - direct).max() <= 1e-13 * np.abs(direct).max()
    halo = PS.poisson_root_isolated(rho, dh, G, halo=2)
    pts = [(-1, 0, 0), (5, 6, 7), (-2, -2, -2), (6, 7, 8), (2, -2, 8)]
    want = PS.pairwise_potential(rho, dh, G, points=pts)
    got = [halo[z + 2, y + 2, x + 2] for z, y, x in pts]
    assert np.abs(np.array(got) - want).max() <= 1e-13 * np.abs(want).max()


def polytrope_error(n, R=0.35, G=1.0):
    """The n = 1 polytrope rho = sin(kr)/(kr) (k = pi/R, zero outside R) in
    the unit box: inside, phi = -(4 pi G / k^2)(1 + sin(kr)/(kr)); outside,
    -G M / r with M = 4 pi^2 / k^3.  Max relative errors of the isolated
    solve for r < R/2 and for r > 0.45."""
    dh = 1.0 / n
    c = (np.arange(n) + 0.5) * dh - 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    k = np.pi / R
    rho = np.where(r < R, np.sinc(k * r / np.pi), 0.0)
    phi = PS.poisson_root_isolated(rho, dh, G)
    exact = np.where(r < R, -(4 * np.pi * G / k ** 2) * (1 + np.sinc(k * r / np.pi)),
                     -G * 4 * np.pi ** 2 / k ** 3 / np.maximum(r, 1e-30))
    inner, outer = r < R / 2, r > 0.45
    return (np.abs(phi - exact)[inner].max() / np.abs(exact[inner]).max(),
            np.abs(phi - exact)[outer].max() / np.abs(exact[outer]).max())


def test_isolated_polytrope_converges_at_second_order():
    e = [polytrope_error(n) for n in (16, 32, 64)]
    assert e[0][0] / e[1][0] > 3.5 and e[1][0] / e[2][0] > 3.5, e  # measured 4.0, 3.9
    assert e[2][0] < 2.5e-3 and e[2][1] < 1e-4, e  # measured 2.2e-3, 4.3e-5


def test_time_interpolated_boundary_is_affine():
    """A refined patch's potential after a fixed number of SOR iterations
    is an affine function of the parent potential (boundary and initial
    guess are linear in it, the density term fixed), so the solve from the
    time-interpolated parent potential equals the same weights applied to
    the two solves."""
    rng = np.random.default_rng(8)
    n = 16
    A_ = rng.random((n, n, n))
    B_ = rng.random((n, n, n))
    rho_c = 1.0 + rng.random((n, n, n))
    rho_f = np.repeat(np.repeat(np.repeat(rho_c, 2, 0), 2, 1), 2, 2) * (1 + 0.1 * rng.random((2 * n,) * 3))
    fmask = np.zeros((2 * n,) * 3, dtype=bool)
    fmask[8:24, 8:24, 8:24] = True
    args = (rho_f, fmask, rho_c, (8, 16, 8), 1.0 / (2 * n), 1.0, 1.6, 10)
    w = 0.3
    mid = PS.refined_patch_potential(PS.time_interp(A_, B_, w), *args)
    a = PS.refined_patch_potential(A_, *args)
    b = PS.refined_patch_potential(B_, *args)
    assert np.abs(mid - ((1 - w) * a + w * b)).max() <= 1e-13 * np.abs(mid).max()
    assert np.array_equal(PS.time_interp(A_, B_, 0.0), A_) and np.array_equal(PS.time_interp(A_, B_, 1.0), B_)


def test_ctu_predictor_with_zero_field_is_the_plain_ctu_step():
    """The CTU variant of the coupling's predictor (the half-step source on
    the normal-predicted states) reduces to the plain CTU step for g = 0,
    and for a uniform state in a constant field, as the MUSCL-Hancock one,
    leaves the state unchanged (the source enters only through the fluxes
    of equal face states)."""
    import oracle
    from paper_1712_07070_b300 import ics
    U = ics.sod_noise(16, seed=6, gamma=G53)
    with oracle.scheme(ctu=True):
        dt = oracle.dt_cfl(U, G53, 0.5, 1 / 16)
        a, _ = oracle.step_periodic(U, 1 / 16, dt, G53)
        b, _ = oracle.step_gravity_predictor(U, np.zeros((3,) + U.shape[1:]), 1 / 16, dt, G53)
        assert np.array_equal(a, b)
        V = np.zeros((5, 4, 4, 4))
        V[0], V[1], V[4] = 1.3, 0.2, 2.0
        g = np.broadcast_to(np.array([0.3, 0.5, -0.2])[:, None, None, None], (3, 4, 4, 4)).copy()
        c, _ = oracle.step_gravity_predictor(V, g, 1 / 4, 0.01, G53)
        assert np.array_equal(c, V)
