"""Plain numpy oracle of GAMER-2's gravity solvers (section 2.3 Gravity and
section 3.1 / Appendix A for the refined-level solver).

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Readings taken (the paper names the methods; their details are ours):
  * root level, periodic: the discretised Poisson equation with the
    second-order (7-point) finite-difference Laplacian,
        sum_d (phi_{i+e_d} - 2 phi_i + phi_{i-e_d}) / dh^2 = 4 pi G (rho_i - <rho>),
    solved by FFT: phi_k = 4 pi G rho_k dh^2 / lambda_k with
    lambda_k = -2 sum_d (1 - cos(2 pi k_d / N_d)), phi_0 = 0;
  * refined levels: every patch is solved on its own (8 + 2*5)^3 = 18^3 grid
    (5 buffer cells per side); the outermost layer of the grid is fixed
    during the iterations.  Its values and the initial guess of the whole
    grid come from the coarse potential by quadratic interpolation in space,
    taken as the tensor product of the 1-D quadratic through the coarse
    cells c-1, c, c+1 evaluated at the child's offset x = -1/4 or +1/4
    (coarse-cell units):  phi_c + x (phi_{c+1} - phi_{c-1}) / 2
                           + x^2 (phi_{c+1} - 2 phi_c + phi_{c-1}) / 2,
    applied along x, then y, then z;
  * the density on the 18^3 grid is the fine level's where a fine patch
    holds the cell, else the coarse cell's (injection);
  * SOR (Press et al. 2007): red-black ordering (red: i+j+k even in the
    18^3 grid's indices), one sweep of red then black cells is an
    iteration, each interior cell
        phi += omega (sum of 6 neighbours - 6 phi - dh^2 4 pi G rho) / 6,
    a fixed number of iterations;
  * with adaptive time steps the parent's potential at the child's time is
    linear in time between its two potentials, taken per coarse cell
    before the spatial interpolation: (1 - w) phi_old + w phi_new;
  * acceleration g = -grad phi at cell centres by two-point
    (phi_{i+1} - phi_{i-1}) / (2 dh) or four-point
    (-phi_{i+2} + 8 phi_{i+1} - 8 phi_{i-1} + phi_{i-2}) / (12 dh)
    central differences.
  * root level, isolated: every cell is a point mass m = rho dh^3 at its
    centre and the potential is the pairwise sum over the other cells,
        phi_i = -G sum_{j != i} m_j / |r_i - r_j|,
    evaluated by a cyclic FFT convolution on a zero-padded grid of at
    least 2 N + 4 cells per axis (a multiple of 2, 3, 5, 7 only), which is
    exact for offsets up to N + 1 and so also gives phi on the two layers
    outside the box that the accelerations of the edge cells need.
Arrays are [z][y][x] (x fastest) like the hydro oracle's.
"""
import numpy as np

FOUR_PI = 4.0 * np.pi


def poisson_root_periodic(rho, dh, G=1.0):
    """Periodic FFT solution of the 7-point Poisson equation on the root grid."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    src = FOUR_PI * G * (rho - rho.mean()) * dh * dh
    sk = np.fft.rfftn(src)
    kz = np.arange(nz)[:, None, None]
    ky = np.arange(ny)[None, :, None]
    kx = np.arange(nx // 2 + 1)[None, None, :]
    lam = -2.0 * ((1 - np.cos(2 * np.pi * kx / nx)) + (1 - np.cos(2 * np.pi * ky / ny)) +
                  (1 - np.cos(2 * np.pi * kz / nz)))
    lam[0, 0, 0] = 1.0
    pk = sk / lam
    pk[0, 0, 0] = 0.0
    return np.fft.irfftn(pk, s=(nz, ny, nx), axes=(0, 1, 2))


def laplacian_periodic(phi, dh):
    """The 7-point discrete Laplacian with periodic wrap."""
    out = -6.0 * phi
    for ax in range(3):
        out = out + np.roll(phi, 1, axis=ax) + np.roll(phi, -1, axis=ax)
    return out / (dh * dh)


def quad1d(pm, p0, pp, x):
    """The quadratic through (-1, pm), (0, p0), (1, pp) at x."""
    return p0 + x * (pp - pm) / 2.0 + x * x * (pp - 2.0 * p0 + pm) / 2.0


def interp_quadratic(phi_c, fx, fy, fz):
    """Quadratic interpolation of the periodic coarse field phi_c at the fine
    cells with integer fine indices (fx, fy, fz) (1-D index arrays, any
    range: periodic on the fine grid of twice the coarse size).  Returns
    [len(fz)][len(fy)][len(fx)]."""
    nzc, nyc, nxc = phi_c.shape

    def split(f, n):
        f = np.asarray(f) % (2 * n)
        return f // 2, np.where(f % 2 == 0, -0.25, 0.25)

    cx, ox = split(fx, nxc)
    cy, oy = split(fy, nyc)
    cz, oz = split(fz, nzc)
    # along x on the 3 x 3 coarse (z, y) neighbourhoods of every needed coarse row
    zz = (cz[:, None] + np.arange(-1, 2)[None, :]) % nzc       # [nfz][3]
    yy = (cy[:, None] + np.arange(-1, 2)[None, :]) % nyc       # [nfy][3]
    xx = (cx[:, None] + np.arange(-1, 2)[None, :]) % nxc       # [nfx][3]
    A = phi_c[zz[:, :, None, None, None, None], yy[None, None, :, :, None, None], xx[None, None, None, None, :, :]]
    # A: [nfz][3][nfy][3][nfx][3]
    X = quad1d(A[..., 0], A[..., 1], A[..., 2], ox[None, None, None, None, :])     # [nfz][3][nfy][3][nfx]
    Y = quad1d(X[:, :, :, 0], X[:, :, :, 1], X[:, :, :, 2], oy[None, None, :, None])  # [nfz][3][nfy][nfx]
    Z = quad1d(Y[:, 0], Y[:, 1], Y[:, 2], oz[:, None, None])                         # [nfz][nfy][nfx]
    return Z


def time_interp(phi_old, phi_new, w):
    """The parent's potential at w = (t - t_old) / (t_new - t_old)."""
    return (1.0 - w) * np.asarray(phi_old) + w * np.asarray(phi_new)


def sor(phi0, rho, dh, G, omega, iters):
    """Red-black SOR on a grid whose outermost layer is fixed."""
    phi = np.array(phi0, dtype=np.float64, copy=True)
    n = phi.shape
    k, j, i = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    inner = (k > 0) & (k < n[0] - 1) & (j > 0) & (j < n[1] - 1) & (i > 0) & (i < n[2] - 1)
    red = inner & ((i + j + k) % 2 == 0)
    black = inner & ((i + j + k) % 2 == 1)
    src = dh * dh * FOUR_PI * G * rho
    for _ in range(iters):
        for mask in (red, black):
            nb = (np.roll(phi, 1, 0) + np.roll(phi, -1, 0) + np.roll(phi, 1, 1) + np.roll(phi, -1, 1) +
                  np.roll(phi, 1, 2) + np.roll(phi, -1, 2))
            upd = phi + omega * (nb - 6.0 * phi - src) / 6.0
            phi = np.where(mask, upd, phi)
    return phi


def accel(phi, dh, order=2):
    """g = -grad phi by central differences on the interior of phi's grid:
    returns [3][...] (x, y, z components) on the cells order/2 away from
    every edge of phi."""
    h = order // 2
    sl = tuple(slice(h, s - h) for s in phi.shape)
    out = []
    for ax in (2, 1, 0):  # x, y, z
        def sh(k):
            idx = list(sl)
            s = sl[ax]
            idx[ax] = slice(s.start + k, s.stop + k)
            return phi[tuple(idx)]
        if order == 2:
            d = (sh(1) - sh(-1)) / (2 * dh)
        else:
            d = (-sh(2) + 8 * sh(1) - 8 * sh(-1) + sh(-2)) / (12 * dh)
        out.append(-d)
    return np.stack(out)


def patch_grid(corner, nbuf=5, n=8):
    """The fine indices of a patch's (n + 2 nbuf)^3 grid along one axis."""
    return np.arange(corner - nbuf, corner + n + nbuf)


def refined_patch_potential(phi_c, rho_f_dense, fmask_dense, rho_c, corner, dh_f, G, omega, iters, nbuf=5):
    """The potential of one refined patch with lower corner (x, y, z) (fine
    indices): density on the patch's grid from the fine level where
    fmask_dense marks a fine cell, else the coarse cell's; boundary and
    initial guess by quadratic interpolation of phi_c; SOR; returns the
    whole (8 + 2 nbuf)^3 grid."""
    gx, gy, gz = (patch_grid(c, nbuf) for c in corner)
    nzf, nyf, nxf = rho_f_dense.shape
    zi, yi, xi = np.ix_(gz % nzf, gy % nyf, gx % nxf)
    rho = np.where(fmask_dense[zi, yi, xi], rho_f_dense[zi, yi, xi],
                   rho_c[(gz % nzf)[:, None, None] // 2, (gy % nyf)[None, :, None] // 2,
                         (gx % nxf)[None, None, :] // 2])
    phi0 = interp_quadratic(phi_c, gx, gy, gz)
    return sor(phi0, rho, dh_f, G, omega, iters)


def accel_periodic(phi, dh, order=2):
    """-grad phi of a periodic field, on every cell."""
    h = order // 2
    return accel(np.pad(phi, h, mode="wrap"), dh, order)


def dt_acc(g, dh, c_acc):
    """Eq. (acc): C_acc (dh / max over cells of max(|a_x|, |a_y|, |a_z|))^(1/2)."""
    return c_acc * np.sqrt(dh / np.abs(g).max())


def step_gravity(U, g_n, dh, dt, gamma, G, order=2, isolated=False):
    """One coupled hydro + self-gravity step on a periodic root grid
    (section 2.3, after Muller & Steinmetz 1995): the predictor (the
    MUSCL-Hancock step with gravity in its half step, hydro_oracle.c), the
    FFT potential and acceleration g^{n+1} of the predicted density, then
    m^{n+1} = m* + (dt/2)(rho^n g^n + rho^{n+1} g^{n+1}) and
    E^{n+1} = E* + (dt/2)(m^n.g^n + m^{n+1}.g^{n+1}).
    isolated: the root potential with isolated boundaries (the hydro stays
    periodic).  Returns (U^{n+1}, phi^{n+1}, g^{n+1}, nbad of the predictor)."""
    import oracle
    Us, nbad = oracle.step_gravity_predictor(U, g_n, dh, dt, gamma)
    if isolated:
        phi = poisson_root_isolated(Us[0], dh, G)
        g1 = accel_isolated(Us[0], dh, G, order)
    else:
        phi = poisson_root_periodic(Us[0], dh, G)
        g1 = accel_periodic(phi, dh, order)
    return gravity_correct(U, g_n, Us, g1, dt), phi, g1, nbad


def gravity_correct(U, g_n, Us, g1, dt):
    """The corrector: momentum from the accelerations at both ends of the
    step, then energy with the corrected momentum."""
    out = Us.copy()
    for d in range(3):
        out[1 + d] = Us[1 + d] + 0.5 * dt * (U[0] * g_n[d] + Us[0] * g1[d])
    out[4] = Us[4] + 0.5 * dt * ((U[1] * g_n[0] + U[2] * g_n[1] + U[3] * g_n[2]) +
                                 (out[1] * g1[0] + out[2] * g1[1] + out[3] * g1[2]))
    return out


def pairwise_potential(rho, dh, G=1.0, points=None):
    """Isolated potential by direct summation over all cell pairs (small
    grids): at the cell centres, or at the given (z, y, x) cell-index
    points (any integers, inside or outside the box)."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    src = np.stack([z.ravel(), y.ravel(), x.ravel()], axis=1).astype(np.float64)
    m = rho.ravel() * dh ** 3
    pts = src if points is None else np.asarray(points, dtype=np.float64)
    out = np.empty(len(pts))
    for i, p in enumerate(pts):
        r = np.sqrt(((src - p) ** 2).sum(axis=1)) * dh
        nz_ = r > 0
        out[i] = -G * (m[nz_] / r[nz_]).sum()
    return out.reshape(rho.shape) if points is None else out


def smooth7(n):
    """The smallest integer >= n whose prime factors are 2, 3, 5 or 7."""
    while True:
        k = n
        for p in (2, 3, 5, 7):
            while k % p == 0:
                k //= p
        if k == 1:
            return n
        n += 1


def isolated_sizes(shape):
    """The padded grid of the isolated solve, per axis (z, y, x)."""
    return tuple(smooth7(2 * n + 4) for n in shape)


def poisson_root_isolated(rho, dh, G=1.0, halo=0):
    """Isolated potential of the root grid by zero-padded FFT convolution
    with the point-mass kernel -G dh^2 / |offset in cells| (0 at offset 0).
    halo > 0 (at most 2): also the layers outside the box, returned as an
    array of shape N + 2 halo per axis."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape
    M = isolated_sizes(n)
    pad = np.zeros(M)
    pad[:n[0], :n[1], :n[2]] = rho
    offs = [np.where(np.arange(m) <= m // 2, np.arange(m), np.arange(m) - m) for m in M]
    dz, dy, dx = np.meshgrid(*offs, indexing="ij")
    d = np.sqrt(dx * dx + dy * dy + dz * dz)
    g = np.zeros(M)
    g[d > 0] = -G * dh * dh / d[d > 0]
    phi = np.fft.irfftn(np.fft.rfftn(pad) * np.fft.rfftn(g), s=M, axes=(0, 1, 2))
    idx = [np.arange(-halo, k + halo) % m for k, m in zip(n, M)]
    return phi[np.ix_(*idx)]


def accel_isolated(rho, dh, G=1.0, order=2):
    """-grad phi of the isolated potential on every cell of the box."""
    h = order // 2
    return accel(poisson_root_isolated(rho, dh, G, halo=h), dh, order)
