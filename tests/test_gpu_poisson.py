"""GPU parity of the gravity solvers (section 2.3; Appendix A) against the
numpy oracle (oracle/poisson.py): the root level's periodic FFT potential
and its accelerations (two- and four-point), and the refined levels' SOR
potential on 18^3 grids per patch (density from the level or injected from
its parent, boundary and initial guess by quadratic interpolation of the
parent's potential) on a three-level hierarchy, each level's oracle input
being the oracle's own potential of the level above."""
import numpy as np
import pytest

from oracle import poisson as PS
from oracle.amr import OracleHierarchy, cell_mask
from paper_1712_07070_b300 import amr_hydro as A
from paper_1712_07070_b300 import ics
from test_gpu_amr import compare

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0


def dense_of(slots, corners, shape):
    out = np.zeros(shape)
    for s, (x, y, z) in enumerate(corners):
        out[..., z:z + 8, y:y + 8, x:x + 8] = slots[s]
    return out


# FP32 transforms (the FP32-compute mode): an FFT of N values in precision
# eps carries a round-off of about eps log2(N) of the transformed vector's
# norm (eps 6e-8, log2(N) 17 here: 1e-6); the inverse Laplacian damps it,
# and a difference over 2 dh raises it against the smooth part of g by at
# most N_x / (2 pi) (5 at 32 cells): bounds 1e-5 of max|phi|, 1e-4 of max|g|.
ROOT_TOL = {A.AMR_FP64: (1e-12, 1e-11), A.AMR_FP32_ACC64: (1e-5, 1e-4)}


@pytest.mark.parametrize("prec", [A.AMR_FP64, A.AMR_FP32_ACC64])
@pytest.mark.parametrize("order", [2, 4])
def test_root_periodic_fft(order, prec):
    import torch
    from paper_1712_07070_b300.uniform import UniformGrid
    nx, ny, nz = 32, 48, 64
    U0 = ics.sod_noise(nx, seed=17, ny=ny, nz=nz)
    g = UniformGrid((nx, ny, nz), prec=prec)
    g.upload(U0)
    n = g.n_patches
    phi = torch.zeros((n, 8, 8, 8), dtype=torch.float64, device="cuda")
    acc = torch.zeros((n, 3, 8, 8, 8), dtype=torch.float64, device="cuda")
    A.amr_hydro_poisson_root(g.ctx, 0.9, phi, acc, order)
    corners = g.tables[0].cpu().numpy()
    ph = dense_of(phi.cpu().numpy(), corners, (nz, ny, nx))
    ac = dense_of(acc.cpu().numpy(), corners, (3, nz, ny, nx))
    g.close()
    dh = 1.0 / nx
    ref = PS.poisson_root_periodic(U0[0], dh, 0.9)
    tp, tg = ROOT_TOL[prec]
    assert np.abs(ph - ref).max() <= tp * np.abs(ref).max()
    h = order // 2
    gref = PS.accel(np.pad(ref, h, mode="wrap"), dh, order)
    assert np.abs(ac - gref).max() <= tg * np.abs(gref).max()


# FP32 SOR (the FP32-compute mode): every sweep rounds phi to eps_32 = 6e-8
# of its size and the error iteration contracts, so the iterate stays
# within a few eps / (1 - rho_SOR) of the FP64 one (rho_SOR < 0.9 here):
# 1e-5 of max|phi|; the four-point difference (weights summing to 18/12)
# over dh raises that against max|g| by |phi| / (|g| dh), about 20 for these
# blobs: 3e-4 of max|g|.
SOR_TOL = {A.AMR_FP64: (1e-12, 1e-10), A.AMR_FP32_ACC64: (1e-5, 3e-4)}


@pytest.mark.parametrize("prec", [A.AMR_FP64, A.AMR_FP32_ACC64])
def test_refined_levels_sor(prec):
    import torch
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(32, seed=3)
    H = AmrHierarchy(U0, lmax=2, theta=0.05, nbuf=(8, 4), max_patches=6000, prec=prec)
    O = OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8, 4])
    compare(H, O, 1e-12)  # the same patches and states on every level
    G, omega, iters = 1.0, 1.7, 40
    phis = []
    n0 = H.n_patches(0)
    phi = torch.zeros((n0, 8, 8, 8), dtype=torch.float64, device="cuda")
    A.amr_hydro_poisson_root(H.ctx, G, phi)
    phis.append(phi)
    accs = [None]
    for l in (1, 2):
        n = H.n_patches(l)
        phi = torch.zeros((max(n, 1), 8, 8, 8), dtype=torch.float64, device="cuda")
        acc = torch.zeros((max(n, 1), 3, 8, 8, 8), dtype=torch.float64, device="cuda")
        A.amr_hydro_poisson_level(H.ctx, l, G, omega, iters, phis[-1], phi, acc, 4)
        phis.append(phi)
        accs.append(acc)
    torch.cuda.synchronize()
    # the oracle, each level from its own potential of the level above
    phic = PS.poisson_root_periodic(O.lv[0].U[0], 1.0 / 32, G)
    checked = 0
    for l in (1, 2):
        Lo, Lc = O.lv[l], O.lv[l - 1]
        fmask = cell_mask(Lo.mask)
        dh = 1.0 / (32 << l)
        phi_l = np.zeros(Lo.U[0].shape)
        gp, ga = phis[l].cpu().numpy(), accs[l].cpu().numpy()
        for s, (x, y, z) in enumerate(H.corners(l)):
            grid = PS.refined_patch_potential(phic, Lo.U[0], fmask, Lc.U[0], (x, y, z), dh, G, omega, iters)
            act = grid[5:13, 5:13, 5:13]
            tp, tg = SOR_TOL[prec]
            assert np.abs(gp[s] - act).max() <= tp * np.abs(act).max(), (l, s)
            gref = PS.accel(grid, dh, 4)[:, 3:11, 3:11, 3:11]
            assert np.abs(ga[s] - gref).max() <= tg * np.abs(gref).max(), (l, s)
            phi_l[z:z + 8, y:y + 8, x:x + 8] = act
            checked += 1
        phic = phi_l
    assert checked > 100
    H.close()


def gravity_ics(n, seed):
    """A self-gravitating box: the density blobs of the hydro tests (contrast
    30, Mach 1.5) whose potential wells drive them inwards."""
    return ics.blobs(n, seed=seed, contrast=30.0, mach=1.5)


@pytest.mark.parametrize("prec,tol,c_acc", [(A.AMR_FP64, 1e-12, 0.0), (A.AMR_FP32_ACC64, 1e-5, 0.0),
                                            (A.AMR_FP64, 1e-12, 0.05)])
@pytest.mark.parametrize("order", [2, 4])
def test_coupled_gravity_step(prec, tol, c_acc, order):
    """Hydro + self-gravity steps (the gravity predictor in the MUSCL-Hancock
    half step, the FFT potential of the predicted density, the corrector)
    against the oracle's, state, potential and acceleration, with the CFL dt
    taken on the device (c_acc 0.05: Eq. (acc) binds, about 0.65 of the CFL
    dt here)."""
    from paper_1712_07070_b300.uniform import UniformGrid
    n, G = 32, 2.0
    U = gravity_ics(n, 5)
    g = UniformGrid((n, n, n), prec=prec)
    g.upload(U)
    _, acc = g.gravity(G, order)
    dh = 1.0 / n
    gref = PS.accel_periodic(PS.poisson_root_periodic(U[0], dh, G), dh, order)
    assert np.abs(g.to_dense(acc) - gref).max() <= ROOT_TOL[prec][1] * np.abs(gref).max()
    import oracle
    t = 0.0
    for _ in range(3):
        dt = oracle.dt_cfl2(U, G53, 0.5, dh)
        if c_acc:
            assert PS.dt_acc(gref, dh, c_acc) < 0.8 * dt
            dt = PS.dt_acc(gref, dh, c_acc)
        # FP64: the device's own CFL dt; FP32: the oracle's (the FP32 speed differs in the last bits)
        phi, acc = g.step_gravity(G, acc, -1.0 if prec == A.AMR_FP64 else dt, order, c_acc)
        U, phir, gref, nbad = PS.step_gravity(U, gref, dh, dt, G53, G, order)
        assert nbad == 0
        t += dt
        assert g.time() == pytest.approx(t, rel=1e-12)
        V = g.download()
        scale = np.abs(U).reshape(5, -1).max(axis=1)
        err = (np.abs(V - U).reshape(5, -1).max(axis=1) / scale).max()
        assert err <= tol, err
        if prec == A.AMR_FP32_ACC64:  # continue from the GPU's own state
            U = V
            gref = PS.accel_periodic(PS.poisson_root_periodic(U[0], dh, G), dh, order)
            g.upload(U)
            _, acc = g.gravity(G, order)
        else:
            assert np.abs(g.to_dense(phi) - phir).max() <= 1e-12 * np.abs(phir).max()
            assert np.abs(g.to_dense(acc) - gref).max() <= 1e-11 * np.abs(gref).max()
    g.close()


def test_coupled_gravity_rejects_other_schemes():
    import torch
    from paper_1712_07070_b300.uniform import UniformGrid
    for sch in ({"scheme": A.AMR_SCHEME_VL}, {"recon": A.AMR_RECON_PPM}):
        g = UniformGrid((16, 16, 16), scheme=sch)
        g.upload(ics.blobs(16, seed=1))
        acc = torch.zeros((g.n_patches, 3, 8, 8, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(A.AmrHydroError):
            g.step_gravity(1.0, acc)
        g.close()


@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 5e-5)])
def test_coupled_gravity_step_ctu(prec, tol):
    """The coupling with the CTU scheme (the half-step source on the normal-
    predicted face states; Eq. (CFL1) time step taken on the device in
    FP64), three steps against the oracle; FP32 compute at the CTU scheme's
    derived per-step bound."""
    import oracle
    from paper_1712_07070_b300.uniform import UniformGrid
    n, G = 32, 2.0
    U = gravity_ics(n, 5)
    g = UniformGrid((n, n, n), prec=prec, scheme={"scheme": A.AMR_SCHEME_CTU})
    g.upload(U)
    dh = 1.0 / n
    _, acc = g.gravity(G, 2)
    gref = PS.accel_periodic(PS.poisson_root_periodic(U[0], dh, G), dh, 2)
    t = 0.0
    with oracle.scheme(ctu=True):
        for _ in range(3):
            dt = oracle.dt_cfl(U, G53, 0.5, dh)
            phi, acc = g.step_gravity(G, acc, -1.0 if prec == A.AMR_FP64 else dt, 2)
            U, phir, gref, nbad = PS.step_gravity(U, gref, dh, dt, G53, G, 2)
            assert nbad == 0
            t += dt
            assert g.time() == pytest.approx(t, rel=1e-12)
            V = g.download()
            scale = np.abs(U).reshape(5, -1).max(axis=1)
            err = (np.abs(V - U).reshape(5, -1).max(axis=1) / scale).max()
            assert err <= tol, err
            if prec == A.AMR_FP32_ACC64:  # continue from the GPU's own state
                U = V
                gref = PS.accel_periodic(PS.poisson_root_periodic(U[0], dh, G), dh, 2)
                g.upload(U)
                _, acc = g.gravity(G, 2)
    g.close()


# Isolated boundaries in FP32: the same eps log2(N) round-off, now of a
# potential dominated by its smooth -GM/r part; a difference over 2 dh
# raises it against max|g| ~ GM/L^2 by about N (64 here): 1e-5 of max|phi|,
# 5e-4 of max|g|.
ISO_TOL = {A.AMR_FP64: (1e-12, 1e-11), A.AMR_FP32_ACC64: (1e-5, 5e-4)}


@pytest.mark.parametrize("prec", [A.AMR_FP64, A.AMR_FP32_ACC64])
@pytest.mark.parametrize("order", [2, 4])
def test_root_isolated(order, prec):
    """Isolated root potential (every cell a point mass, the pairwise sum by
    zero-padded FFT) and its accelerations, the edge cells' differences
    reaching the two layers outside the box, on a 32 x 48 x 64 grid (padded
    to 70 x 100 x 135), twice on one context (the kernel's transform is
    made once)."""
    import torch
    from paper_1712_07070_b300.uniform import UniformGrid
    nx, ny, nz = 32, 48, 64
    U0 = ics.sod_noise(nx, seed=19, ny=ny, nz=nz)
    g = UniformGrid((nx, ny, nz), prec=prec, scheme={"gravity_bc": A.AMR_GRAVITY_ISOLATED})
    g.upload(U0)
    dh = 1.0 / nx
    ref = PS.poisson_root_isolated(U0[0], dh, 0.7)
    gref = PS.accel_isolated(U0[0], dh, 0.7, order)
    tp, tg = ISO_TOL[prec]
    for _ in range(2):
        phi, acc = g.gravity(0.7, order)
        ph, ac = g.to_dense(phi), g.to_dense(acc)
        assert np.abs(ph - ref).max() <= tp * np.abs(ref).max()
        assert np.abs(ac - gref).max() <= tg * np.abs(gref).max()
    g.close()


def test_coupled_gravity_step_isolated():
    """Two coupled steps with the isolated root potential, FP64, against the
    oracle at 1e-12."""
    from paper_1712_07070_b300.uniform import UniformGrid
    import oracle
    n, G = 32, 2.0
    U = gravity_ics(n, 7)
    g = UniformGrid((n, n, n), scheme={"gravity_bc": A.AMR_GRAVITY_ISOLATED})
    g.upload(U)
    dh = 1.0 / n
    _, acc = g.gravity(G, 2)
    gref = PS.accel_isolated(U[0], dh, G, 2)
    for _ in range(2):
        dt = oracle.dt_cfl2(U, G53, 0.5, dh)
        phi, acc = g.step_gravity(G, acc, dt, 2)
        U, phir, gref, nbad = PS.step_gravity(U, gref, dh, dt, G53, G, 2, isolated=True)
        assert nbad == 0
        V = g.download()
        scale = np.abs(U).reshape(5, -1).max(axis=1)
        assert (np.abs(V - U).reshape(5, -1).max(axis=1) / scale).max() <= 1e-12
        assert np.abs(g.to_dense(phi) - phir).max() <= 1e-12 * np.abs(phir).max()
        assert np.abs(g.to_dense(acc) - gref).max() <= 1e-11 * np.abs(gref).max()
    g.close()


def test_refined_level_sor_time_interpolated():
    """The refined-level solve with the parent's potential interpolated in
    time (w = 0.3 between two parent potentials), FP64, against the oracle
    at 1e-12 on every level-1 patch of the blob hierarchy."""
    import torch
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(32, seed=3)
    H = AmrHierarchy(U0, lmax=1, theta=0.05, nbuf=(8,), max_patches=6000)
    O = OracleHierarchy(U0, lmax=1, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8])
    compare(H, O, 1e-12)
    G, omega, iters, w = 1.0, 1.7, 30, 0.3
    c = (np.arange(32) + 0.5) / 32
    old = PS.poisson_root_periodic(O.lv[0].U[0], 1.0 / 32, G)
    new = 0.8 * old + 0.05 * np.sin(2 * np.pi * c)[None, None, :] * np.cos(2 * np.pi * c)[:, None, None]

    def slots(dense):
        return torch.from_numpy(np.stack([dense[z:z + 8, y:y + 8, x:x + 8] for x, y, z in H.corners(0)])).cuda()

    n1 = H.n_patches(1)
    phi = torch.zeros((n1, 8, 8, 8), dtype=torch.float64, device="cuda")
    acc = torch.zeros((n1, 3, 8, 8, 8), dtype=torch.float64, device="cuda")
    A.amr_hydro_poisson_level_t(H.ctx, 1, G, omega, iters, slots(old), slots(new), w, phi, acc, 2)
    gp, ga = phi.cpu().numpy(), acc.cpu().numpy()
    Lo, Lc = O.lv[1], O.lv[0]
    fmask = cell_mask(Lo.mask)
    dh = 1.0 / 64
    phic = PS.time_interp(old, new, w)
    for s, (x, y, z) in enumerate(H.corners(1)):
        grid = PS.refined_patch_potential(phic, Lo.U[0], fmask, Lc.U[0], (x, y, z), dh, G, omega, iters)
        act = grid[5:13, 5:13, 5:13]
        assert np.abs(gp[s] - act).max() <= 1e-12 * np.abs(act).max(), s
        gref = PS.accel(grid, dh, 2)[:, 4:12, 4:12, 4:12]
        assert np.abs(ga[s] - gref).max() <= 1e-10 * np.abs(gref).max(), s
    with pytest.raises(A.AmrHydroError):
        A.amr_hydro_poisson_level_t(H.ctx, 1, G, omega, iters, slots(old), slots(new), 1.5, phi, acc, 2)
    H.close()


def test_gravity_edge_cases():
    """Zero SOR iterations give the interpolated initial guess; no
    acceleration array; invalid arguments are rejected without a launch."""
    import torch
    from paper_1712_07070_b300.amr import AmrHierarchy
    from paper_1712_07070_b300.uniform import UniformGrid
    U0 = ics.blobs(32, seed=3)
    H = AmrHierarchy(U0, lmax=1, theta=0.05, nbuf=(8,), max_patches=6000)
    O = OracleHierarchy(U0, lmax=1, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8])
    compare(H, O, 1e-12)
    phi0 = torch.zeros((H.n_patches(0), 8, 8, 8), dtype=torch.float64, device="cuda")
    A.amr_hydro_poisson_root(H.ctx, 1.0, phi0)  # no acceleration array
    n1 = H.n_patches(1)
    phi1 = torch.zeros((n1, 8, 8, 8), dtype=torch.float64, device="cuda")
    A.amr_hydro_poisson_level(H.ctx, 1, 1.0, 1.7, 0, phi0, phi1)
    phic = PS.poisson_root_periodic(O.lv[0].U[0], 1.0 / 32, 1.0)
    fmask = cell_mask(O.lv[1].mask)
    got = phi1.cpu().numpy()
    for s, (x, y, z) in enumerate(H.corners(1)):
        grid = PS.refined_patch_potential(phic, O.lv[1].U[0], fmask, O.lv[0].U[0], (x, y, z), 1.0 / 64, 1.0, 1.7, 0)
        assert np.abs(got[s] - grid[5:13, 5:13, 5:13]).max() <= 1e-12 * np.abs(grid).max(), s
    with pytest.raises(A.AmrHydroError):  # the output may not overwrite the parent potential
        A.amr_hydro_poisson_level(H.ctx, 1, 1.0, 1.7, 10, phi0, phi0)
    for bad in (dict(iters=-1), dict(acc_order=3), dict(level=2)):
        kw = dict(level=1, iters=10, acc_order=2)
        kw.update(bad)
        with pytest.raises(A.AmrHydroError):
            A.amr_hydro_poisson_level(H.ctx, kw["level"], 1.0, 1.7, kw["iters"], phi0, phi1, phi1, kw["acc_order"])
    H.close()
    g = UniformGrid((16, 16, 16))
    g.upload(ics.blobs(16, seed=1))
    _, acc = g.gravity(1.0, 2)
    for kw in (dict(c_acc=-1.0), dict(order=3), dict(dt=float("nan"))):
        args = dict(dt=-1.0, order=2, c_acc=0.0)
        args.update(kw)
        with pytest.raises(A.AmrHydroError):
            g.step_gravity(1.0, acc, args["dt"], args["order"], args["c_acc"])
    phi = torch.zeros((g.n_patches, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(A.AmrHydroError):  # the new acceleration may not overwrite g^n
        A.amr_hydro_advance_gravity(g.ctx, -1.0, 1.0, acc, phi, acc, 2)
    acc2 = torch.zeros_like(acc)
    with pytest.raises(A.AmrHydroError):  # nor may the new potential (it is written before the corrector)
        A.amr_hydro_advance_gravity(g.ctx, -1.0, 1.0, acc, acc.view(-1)[:phi.numel()].view_as(phi), acc2, 2)
    with pytest.raises(A.AmrHydroError):  # nor the level's state
        A.amr_hydro_advance_gravity(g.ctx, -1.0, 1.0, acc, g.state().view(-1)[:phi.numel()].view_as(phi), acc2, 2)
    g.close()


def test_root_solves_at_the_benchmark_size():
    """The 256^3 root solves of the benchmark, in its configuration: the
    periodic potential satisfies the 7-point discrete Poisson equation at
    2000 sampled cells (a property at any size); the isolated potential
    equals the direct pairwise sum over all 16.7 M cells at 6 sampled cells
    (corners and centre included)."""
    from paper_1712_07070_b300.uniform import UniformGrid
    n, G = 256, 1.0
    U0 = ics.turbulence(n, seed=1)
    U0[0] *= 1.0 + 0.5 * np.sin(2 * np.pi * (np.arange(n) + 0.5) / n)[None, None, :]  # a density contrast
    dh = 1.0 / n
    rng = np.random.default_rng(11)
    g = UniformGrid((n, n, n))
    g.upload(U0)
    phi, _ = g.gravity(G, 2)
    ph = g.to_dense(phi)
    g.close()
    pts = rng.integers(0, n, size=(2000, 3))
    z, y, x = pts.T
    lap = -6.0 * ph[z, y, x]
    for d in range(3):
        for s in (-1, 1):
            q = pts.copy()
            q[:, d] = (q[:, d] + s) % n
            lap += ph[q[:, 0], q[:, 1], q[:, 2]]
    src = 4 * np.pi * G * (U0[0][z, y, x] - U0[0].mean()) * dh * dh
    assert np.abs(lap - src).max() <= 1e-10 * np.abs(src).max()
    g = UniformGrid((n, n, n), scheme={"gravity_bc": A.AMR_GRAVITY_ISOLATED})
    g.upload(U0)
    phi, _ = g.gravity(G, 2)
    ph = g.to_dense(phi)
    g.close()
    pts = [(0, 0, 0), (255, 255, 255), (128, 128, 128), (0, 255, 17), (200, 3, 90), (31, 140, 255)]
    want = PS.pairwise_potential(U0[0], dh, G, points=pts)
    got = np.array([ph[p] for p in pts])
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("prec", [A.AMR_FP64, A.AMR_FP32_ACC64])
def test_coupled_step_at_the_benchmark_size(prec):
    """Two 256^3 hydro + self-gravity steps as the benchmark runs them (device
    dt): mass is conserved to round-off (gravity changes no density and the
    fluxes are conservative), the time record advances by the device's CFL
    steps, and the new acceleration is the root solve of the new state."""
    from paper_1712_07070_b300.uniform import UniformGrid
    n, G = 256, 1.0
    U0 = ics.turbulence(n, seed=1)
    g = UniformGrid((n, n, n), prec=prec)
    g.upload(U0)
    m0 = U0[0].sum()
    _, acc = g.gravity(G, 2)
    for _ in range(2):
        _, acc = g.step_gravity(G, acc, -1.0, 2)
    V = g.download()
    assert abs(V[0].sum() - m0) <= 1e-12 * m0
    assert np.isfinite(V).all() and V[0].min() > 0
    assert g.time() > 0
    _, acc2 = g.gravity(G, 2)
    assert np.array_equal(acc.cpu().numpy(), acc2.cpu().numpy())
    g.close()


# ---- self-gravity inside the AMR W-cycle ---------------------------------------------------

@pytest.mark.parametrize("prec,tol", [(A.AMR_FP64, 1e-12), (A.AMR_FP32_ACC64, 1e-5)])
def test_wcycle_with_gravity_matches_oracle(prec, tol):
    """Two root steps of the three-level blob hierarchy with self-gravity in
    every level step (section 2.3 coupling on the section 2.1 W-cycle): the
    coupled predictor with ghost accelerations from the coarse level, each
    level's Poisson solve at its step's end (root FFT, refined SOR with the
    parent's potential interpolated in time), the corrector, and the
    re-solve of levels a regrid changed; bit-exact patch lists, every
    level's state, potential and acceleration against the oracle."""
    from oracle.amr_gravity import GravityHierarchy
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(32, seed=5, contrast=10.0, mach=1.0)
    G, omega, iters = 2.0, 1.7, 20
    H = AmrHierarchy(U0, lmax=2, theta=0.3, nbuf=(1, 1), prec=prec, max_patches=6000)
    H.set_gravity(G, omega, iters, 2)
    O = GravityHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1, 1], G=G, omega=omega, iters=iters)
    assert 0 < H.n_patches(1) and H.n_patches(2) > 0
    for _ in range(2):
        H.advance_root()
        O.advance(0)
    compare(H, O, tol)
    for l in range(3):
        phi, acc = (t.cpu().numpy() for t in H.gravity(l))
        num_p = den_p = num_g = den_g = 0.0
        for s, (x, y, z) in enumerate(H.corners(l).tolist()):
            rp = O.lv[l].phi[z:z + 8, y:y + 8, x:x + 8]
            rg = O.lv[l].g[:, z:z + 8, y:y + 8, x:x + 8]
            num_p += np.abs(phi[s] - rp).sum()
            den_p += np.abs(rp).sum()
            num_g += np.abs(acc[s] - rg).sum()
            den_g += np.abs(rg).sum()
        assert num_p <= tol * den_p, (l, num_p / den_p)
        assert num_g <= 10 * tol * den_g, (l, num_g / den_g)
    H.close()


def test_set_gravity_rejects_other_schemes():
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(16, seed=1, contrast=10.0, mach=1.0)
    H = AmrHierarchy(U0, lmax=1, theta=0.3, nbuf=(1,), max_patches=2000,
                     scheme={"scheme": A.AMR_SCHEME_CTU})
    with pytest.raises(A.AmrHydroError):
        H.set_gravity(1.0)
    H.close()
    H = AmrHierarchy(U0, lmax=1, theta=0.3, nbuf=(1,), max_patches=2000)
    for bad in (dict(G=-1.0), dict(omega=2.0), dict(iters=-1), dict(acc_order=3)):
        kw = dict(G=1.0, omega=1.7, iters=10, acc_order=2)
        kw.update(bad)
        with pytest.raises(A.AmrHydroError):
            H.set_gravity(kw["G"], kw["omega"], kw["iters"], kw["acc_order"])
    H.close()
