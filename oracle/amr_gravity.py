"""Oracle of self-gravity on the AMR hierarchy (test infrastructure): the
section 2.3 predictor-corrector coupling inside the section 2.1 W-cycle.

TEST INFRASTRUCTURE ONLY: nothing in the product path may import this module.

Readings taken (the paper gives the operations, not their order on a
hierarchy with adaptive time steps):
  * every level keeps its potential and acceleration at its newest time
    (phi, g) and at its previous time (phi_prev, g_prev);
  * a level step from t to t' = t + dt: the predictor (the MUSCL-Hancock
    step with g^n in its half step, g^n on the coarse-fine ghost cells
    interpolated from the coarse level's g like the conserved variables --
    time first, then the minmod-limited prolongation, with no positivity
    decision); the potential of the predicted density at t' (the root: the
    periodic FFT solve; a refined level: every patch's 18^3 SOR solve with
    the parent's potential interpolated in time at
    w = clamp((t' - t_prev) / (t_new - t_prev), 0, 1), 1 when the parent has
    a single time, and the parent's newest density in the buffer zones);
    its acceleration g^{n+1}; the corrector with g^n and g^{n+1};
  * one Poisson solve per level step (section 2.3): fix-up and restriction
    change the coarse state but not its potential;
  * when a regrid changes a level's patches, that level's potential and
    acceleration are solved again from its new state at its time (the
    parent's potential at that same time), for every patch of the level.
"""
import ctypes

import numpy as np

from . import _ptr
from . import poisson as PS
from .amr import OracleHierarchy, _dims, _i3, _u8, _u8p, amr_lib as _amr_lib, cell_mask

_dp = ctypes.POINTER(ctypes.c_double)
_ready = []


def amr_lib():
    L = _amr_lib()
    if not _ready:
        L.or_step_gravity_predictor_fx.argtypes = [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        L.or_step_gravity_predictor_fx.restype = ctypes.c_int64
        L.or_amr_fill_ghost_field.argtypes = [_dp, _u8p, _i3, _dp, _dp, ctypes.c_double]
        _ready.append(True)
    return L


def _flt(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class GravityHierarchy(OracleHierarchy):
    def __init__(self, U_root, lmax, gamma, cfl, theta, nbuf, G, omega=1.7, iters=60, order=2, **kw):
        self.G, self.omega, self.iters, self.order = float(G), float(omega), int(iters), int(order)
        self._grav = False
        super().__init__(U_root, lmax, gamma, cfl, theta, nbuf, **kw)
        for L in self.lv:
            n = L.N
            L.phi = np.zeros((n[2], n[1], n[0]))
            L.g = np.zeros((3, n[2], n[1], n[0]))
        for l in range(lmax + 1):
            if not self.lv[l].empty:
                self._set_level_gravity(l, *self.solve_level(l, self.lv[l].t, self.lv[l].U[0]))
        self._grav = True

    # ---- potentials ----------------------------------------------------------------

    def parent_weight(self, l, t):
        """The parent's time weight for a solve of level l at time t."""
        c = self.lv[l - 1]
        if c.t == c.t_prev or t >= c.t:
            return 1.0
        return min(max((t - c.t_prev) / (c.t - c.t_prev), 0.0), 1.0)

    def solve_level(self, l, t, rho):
        """Potential and acceleration of level l's present cells at time t
        from the density rho (dense level array)."""
        L = self.lv[l]
        dh = self.dh(l)
        if l == 0:
            phi = PS.poisson_root_periodic(rho, dh, self.G)
            return phi, PS.accel_periodic(phi, dh, self.order)
        c = self.lv[l - 1]
        phic = PS.time_interp(c.phi_prev, c.phi, self.parent_weight(l, t))
        fmask = cell_mask(L.mask)
        phi = np.zeros_like(L.phi)
        g = np.zeros_like(L.g)
        h = self.order // 2
        for x, y, z in self.patch_corners(l):
            grid = PS.refined_patch_potential(phic, rho, fmask, c.U[0], (x, y, z), dh, self.G, self.omega,
                                              self.iters)
            phi[z:z + 8, y:y + 8, x:x + 8] = grid[5:13, 5:13, 5:13]
            g[:, z:z + 8, y:y + 8, x:x + 8] = PS.accel(grid, dh, self.order)[:, 5 - h:13 - h, 5 - h:13 - h,
                                                                               5 - h:13 - h]
        return phi, g

    def _set_level_gravity(self, l, phi, g):
        L = self.lv[l]
        L.phi, L.phi_prev = phi, phi.copy()
        L.g, L.g_prev = g, g.copy()

    def fill_ghost_g(self, l, t):
        """g^n of level l's coarse-fine ghost cells from level l-1's g."""
        c, f = self.lv[l - 1], self.lv[l]
        if c.t == c.t_prev or t == c.t:
            w = 1.0
        else:
            w = (t - c.t_prev) / (c.t - c.t_prev)
        for d in range(3):
            fd = _flt(f.g[d])
            amr_lib().or_amr_fill_ghost_field(_ptr(fd), _u8(f.mask), _dims(f.N), _ptr(_flt(c.g_prev[d])),
                                              _ptr(_flt(c.g[d])), w)
            f.g[d] = fd

    # ---- the coupled level step ---------------------------------------------------------

    def advance_level(self, l, dt):
        L = self.lv[l]
        self.fill_ghost(l, L.t)
        if l > 0:
            self.fill_ghost_g(l, L.t)
        N = L.N
        Us = np.empty_like(L.U)
        FX = np.empty((3, 5, N[2], N[1], N[0]))
        g_n = _flt(L.g)
        nb = amr_lib().or_step_gravity_predictor_fx(_ptr(L.U), _ptr(g_n), _ptr(Us), N[0], N[1], N[2], self.dh(l),
                                                     dt, self.gamma, _ptr(FX))
        if nb < 0:
            raise ValueError("the gravity coupling is built for MUSCL-Hancock")
        pres = self.present(l)
        pred = L.U.copy()
        pred[:, pres] = Us[:, pres]
        phi1, g1 = self.solve_level(l, L.t + dt, pred[0])
        corr = PS.gravity_correct(L.U, g_n, pred, g1, dt)
        new = L.U.copy()
        new[:, pres] = corr[:, pres]
        rho = new[0][pres]
        v2 = (new[1][pres] ** 2 + new[2][pres] ** 2 + new[3][pres] ** 2) / rho
        if not ((rho > 0).all() and (new[4][pres] - 0.5 * v2 > 0).all()):
            raise FloatingPointError(f"unphysical cells on level {l}")
        L.U_prev, L.U = L.U, new
        L.t_prev = L.t
        L.phi_prev, L.phi = L.phi, phi1
        L.g_prev, L.g = g_n, g1
        self.n_updates += int(pres.sum())
        self.log.append((l, dt))
        self._registers(l, FX, dt)

    def _registers(self, l, FX, dt):
        L, N = self.lv[l], self.lv[l].N
        if l > 0:
            from .amr import covered
            c = self.lv[l - 1]
            cov = covered(L.mask, N)
            amr_lib().or_amr_cf_fine_accumulate(_ptr(c.acc), _ptr(FX), _u8(cov), _u8(c.mask), _dims(c.N), dt)
        if l < self.lmax and not self.lv[l + 1].empty:
            from .amr import covered
            cov = covered(self.lv[l + 1].mask, self.lv[l + 1].N)
            amr_lib().or_amr_cf_coarse_store(_ptr(L.cfl), _ptr(FX), _u8(cov), _u8(L.mask), _dims(N), dt)
            L.acc[:] = 0.0

    def regrid(self, l, cell_flags=None):
        before = self.lv[l + 1].mask.copy()
        super().regrid(l, cell_flags)
        F = self.lv[l + 1]
        if self._grav and not np.array_equal(before, F.mask):
            if F.empty:
                self._set_level_gravity(l + 1, np.zeros_like(F.phi), np.zeros_like(F.g))
            else:
                self._set_level_gravity(l + 1, *self.solve_level(l + 1, F.t, F.U[0]))
