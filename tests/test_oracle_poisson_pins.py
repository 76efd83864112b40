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
