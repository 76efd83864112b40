"""Seeded synthetic initial conditions, shared bit for bit by the CUDA path and
the CPU oracle.

This module holds no arithmetic of the hydro method itself: it only draws
random numbers with ``numpy.random.default_rng(seed)`` and turns primitive
initial fields (rho, v, P) into conserved arrays U = (rho, rho v, E) in FP64,
layout ``[5][nz][ny][nx]`` with x fastest.  Cell centres are x_i = (i+1/2)/n
on the unit box.

The workloads stand in for the paper's: the GPU-solver throughput test of
section 4.1 (uniform grids of growing size), and the Kelvin-Helmholtz setup of
section 4.2 (shear layers, rho 1/2, vx -+0.5, P=2.5, gamma=1.4).  The recipes
are stated in the design notes of the repository.
"""
import numpy as np


def conserved(rho, vx, vy, vz, P, gamma):
    """Stack primitive fields into U = (rho, rho vx, rho vy, rho vz, E),
    E = P/(gamma-1) + rho |v|^2 / 2."""
    shape = np.broadcast(rho, vx, vy, vz, P).shape
    U = np.empty((5,) + shape, dtype=np.float64)
    U[0] = rho
    np.multiply(rho, vx, out=U[1])
    np.multiply(rho, vy, out=U[2])
    np.multiply(rho, vz, out=U[3])
    e = U[4]
    np.multiply(vx, vx, out=e)
    e += vy * vy
    e += vz * vz
    e *= rho
    e *= 0.5
    e += P / (gamma - 1.0)
    return U


def centres(n):
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def grid(nx, ny=None, nz=None):
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    z, y, x = np.meshgrid(centres(nz), centres(ny), centres(nx), indexing="ij")
    return x, y, z


def fourier_modes(rng, n_modes=8, kmax=4):
    """n_modes integer wave vectors with 1<=|k|<=kmax drawn uniformly from the
    admissible set, plus phases ~U[0, 2pi)."""
    r = np.arange(-kmax, kmax + 1)
    K = np.array(np.meshgrid(r, r, r, indexing="ij")).reshape(3, -1).T
    kk = np.sqrt((K ** 2).sum(1))
    K = K[(kk >= 1) & (kk <= kmax)]
    ks = K[rng.integers(0, len(K), size=n_modes)]
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    return ks, ph


def mode_sum(x, y, z, ks, ph):
    s = np.zeros_like(x)
    for k, p in zip(ks, ph):
        s += np.cos(2.0 * np.pi * (k[0] * x + k[1] * y + k[2] * z) + p)
    return s


def sod_noise(n=64, seed=1, gamma=5.0 / 3.0, ny=None, nz=None):
    """Sod jump along x (rho 1/0.125, P 1/0.1 at x<0.5 / x>=0.5) with the
    density multiplied by 1+0.05*(8 seeded Fourier modes, |k|<=4) and
    velocities ~N(0, 0.01^2) per cell and component."""
    rng = np.random.default_rng(seed)
    x, y, z = grid(n, ny, nz)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    P = np.where(left, 1.0, 0.1)
    ks, ph = fourier_modes(rng)
    rho = rho * (1.0 + 0.05 * mode_sum(x, y, z, ks, ph))
    v = rng.normal(0.0, 0.01, size=(3,) + x.shape)
    return conserved(rho, v[0], v[1], v[2], P, gamma)


def gaussian_velocity(n, rng, kmin=1.0, kmax=16.0, slope=-4.0, rms=1.0):
    """Gaussian random velocity field: 3D power |v(k)|^2 ~ k^slope on integer
    kmin<=|k|<=kmax, zero elsewhere.  For each component, complex normal
    amplitudes are drawn (in a fixed order) for the modes of the band on the
    half-spectrum kx >= 0 only, and a real inverse FFT makes the field real
    (Hermitian by construction); the field is scaled to a 3D rms |v| of ``rms``."""
    import os
    import scipy.fft
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    iz = np.nonzero(np.abs(k1) <= kmax)[0]
    ix = np.nonzero(kr <= kmax)[0]
    KZ, KY, KX = np.meshgrid(k1[iz], k1[iz], kr[ix], indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    band = (kk >= kmin) & (kk <= kmax)
    amp = kk[band] ** (slope / 2.0)
    sel = np.ix_(iz, iz, ix)
    comps = []
    for _ in range(3):
        spec = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
        blk = np.zeros(kk.shape, dtype=np.complex128)
        blk[band] = (rng.normal(size=amp.size) + 1j * rng.normal(size=amp.size)) * amp
        spec[sel] = blk
        comps.append(scipy.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2), workers=os.cpu_count()))
    v = np.stack(comps)
    ms = sum(float(np.vdot(c, c)) for c in comps) / comps[0].size
    v *= rms / np.sqrt(ms)
    return v


def turbulence(n=256, seed=1, gamma=5.0 / 3.0, rho0=1.0, P0=0.6, density_seed=None, eps=0.01):
    """Decaying turbulence: rho=1, P=0.6 (c_s=1 for gamma=5/3), Gaussian random
    velocity with k^-4 power on 1<=|k|<=16, rms Mach 1.  With ``density_seed``
    the density (and with it the momenta, at fixed v and P) is multiplied by
    1 + eps * (8 seeded Fourier modes, |k|<=4): the perturbed initial state of
    the adjoint workload."""
    rng = np.random.default_rng(seed)
    v = gaussian_velocity(n, rng)
    rho = np.full((n, n, n), rho0)
    if density_seed is not None:
        r2 = np.random.default_rng(density_seed)
        x, y, z = grid(n)
        ks, ph = fourier_modes(r2)
        rho = rho * (1.0 + eps * mode_sum(x, y, z, ks, ph))
    P = np.full((n, n, n), P0)
    return conserved(rho, v[0], v[1], v[2], P, gamma)


def kh_box(n, seed, gamma=1.4):
    """Kelvin-Helmholtz shear layer on a periodic unit box: rho=2, vx=+0.5
    for |y-0.5|<0.25, else rho=1, vx=-0.5; vy = 0.01 sin(2 pi m x + phi) with
    m~U{1..4}, phi~U[0,2pi); vz=0; P=2.5."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 5))
    phi = rng.uniform(0.0, 2.0 * np.pi)
    x, y, z = grid(n)
    inner = np.abs(y - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    vx = np.where(inner, 0.5, -0.5)
    vy = 0.01 * np.sin(2.0 * np.pi * m * x + phi)
    vz = np.zeros_like(x)
    P = np.full_like(x, 2.5)
    return conserved(rho, vx, vy, vz, P, gamma)


KH_SIZES = (32, 48, 64, 96, 128, 192)


def kh_batch_sizes(n_boxes=64, seed=4):
    """Box edge lengths drawn uniformly with replacement from KH_SIZES."""
    rng = np.random.default_rng(seed)
    return [int(KH_SIZES[i]) for i in rng.integers(0, len(KH_SIZES), size=n_boxes)]


def blobs(n=128, seed=3, gamma=5.0 / 3.0, n_blobs=3, sigma=0.05, contrast=100.0, mach=2.0):
    """Uniform medium rho=1, P=1 with n_blobs Gaussian overdensities
    rho = 1 + (contrast-1) sum_b exp(-r_b^2/2 sigma^2) (periodic minimum-image
    r_b) moving at Mach ``mach`` of the ambient sound speed along seeded
    isotropic directions."""
    rng = np.random.default_rng(seed)
    x, y, z = grid(n)
    c_amb = np.sqrt(gamma * 1.0 / 1.0)
    rho = np.ones_like(x)
    vel = np.zeros((3,) + x.shape)
    for _ in range(n_blobs):
        c = rng.uniform(0.0, 1.0, size=3)
        nvec = rng.normal(size=3)
        nvec /= np.linalg.norm(nvec)
        d = [np.mod(q - cq + 0.5, 1.0) - 0.5 for q, cq in zip((x, y, z), c)]
        prof = np.exp(-(d[0] ** 2 + d[1] ** 2 + d[2] ** 2) / (2.0 * sigma ** 2))
        rho += (contrast - 1.0) * prof
        for k in range(3):
            vel[k] += mach * c_amb * nvec[k] * prof
    P = np.ones_like(x)
    return conserved(rho, vel[0], vel[1], vel[2], P, gamma)


def uniform_state(n, rho=1.3, v=(0.3, -0.2, 0.1), P=0.7, gamma=5.0 / 3.0, ny=None, nz=None):
    x, _, _ = grid(n, ny, nz)
    o = np.ones_like(x)
    return conserved(rho * o, v[0] * o, v[1] * o, v[2] * o, P * o, gamma)


def advected_wave(n, direction=(1, 0, 0), amp=0.2, gamma=5.0 / 3.0, ny=None, nz=None, speed=1.0):
    """rho = 1 + amp sin(2 pi k.x) with k = direction, v = speed * direction
    (unnormalised), P = 1: a smooth wave advected without change."""
    x, y, z = grid(n, ny, nz)
    k = np.asarray(direction, dtype=np.float64)
    rho = 1.0 + amp * np.sin(2.0 * np.pi * (k[0] * x + k[1] * y + k[2] * z))
    o = np.ones_like(x)
    return conserved(rho, speed * k[0] * o, speed * k[1] * o, speed * k[2] * o, o, gamma)


def riemann_tube(n, left, right, axis=0, transverse=4, gamma=1.4, x0=0.5):
    """1D Riemann problem along ``axis`` on an n x t x t tube; left/right are
    (rho, u, P) with u along ``axis``.  The tube is periodic, so a second
    discontinuity sits at the wrap; compare only away from it."""
    shape = [transverse] * 3
    shape[2 - axis] = n
    nz, ny, nx = shape
    x, y, z = grid(nx, ny, nz)
    q = (x, y, z)[axis]
    L = q < x0
    rho = np.where(L, left[0], right[0])
    un = np.where(L, left[1], right[1])
    P = np.where(L, left[2], right[2])
    vel = [np.zeros_like(x) for _ in range(3)]
    vel[axis] = un
    return conserved(rho, vel[0], vel[1], vel[2], P, gamma)


def smooth_directions(shape, n_dirs, seed, n_modes=8, kmax=4):
    """n_dirs seeded smooth perturbation directions over all 5 fields, each a
    sum of n_modes Fourier modes with |k|<=kmax, scaled to unit max-norm."""
    rng = np.random.default_rng(seed)
    _, nz, ny, nx = shape
    x, y, z = grid(nx, ny, nz)
    out = np.empty((n_dirs,) + tuple(shape))
    for i in range(n_dirs):
        for v in range(shape[0]):
            ks, ph = fourier_modes(rng, n_modes, kmax)
            out[i, v] = mode_sum(x, y, z, ks, ph)
        out[i] /= np.abs(out[i]).max()
    return out
