"""Oracle AMR hierarchy (test infrastructure): the control flow of GAMER-2's
adaptive time stepping and regridding, with every per-cell operation in C
(hydro_oracle.c, amr_oracle.c).

Paper passages followed:
  * section 2.1: levels of 8^3 patches with refinement ratio 2; proper nesting
    (levels of neighbouring patches differ by at most 1); a patch is flagged if
    any cell is; (1+2 N_buf)^3 - 1 flag buffers around flagged cells; no
    explicit derefinement -- a patch is removed when its parent is not flagged
    and it has no children; refinement only where proper nesting allows; one
    level altered at a time; adaptive time steps advanced as a W-cycle with
    the C_inc / C_dec synchronisation rule of the section's pseudo-code.
  * section 2.2: restriction and coarse-fine flux fix-up at synchronisation.
  * section 2.6: Eq. (CFL2) per level.
  * section 2.2 dual-energy formalism (optional, S_root given): the entropy
    per unit volume S of every level is a conserved density carried through
    the same operations -- the step (or_step_dual_fx), ghost interpolation,
    flux registers and fix-up, restriction, and the data of new patches.

Each level is a dense whole-domain array with a patch mask (see amr_oracle.c).
"""
import ctypes

import numpy as np

from . import lib as _hydro_lib, _ptr, _build

_u8p = ctypes.POINTER(ctypes.c_uint8)
_dp = ctypes.POINTER(ctypes.c_double)
_i3 = ctypes.c_int * 3
_amr = None


def amr_lib():
    global _amr
    if _amr is None:
        L = _hydro_lib()
        for name, args in {
            "or_amr_fill_ghost": [_dp, _u8p, _i3, _dp, _dp, ctypes.c_double],
            "or_amr_covered": [_u8p, _i3, _u8p],
            "or_amr_cf_fine_accumulate": [_dp, _dp, _u8p, _u8p, _i3, ctypes.c_double],
            "or_amr_cf_coarse_store": [_dp, _dp, _u8p, _u8p, _i3, ctypes.c_double],
            "or_amr_fixup": [_dp, _dp, _dp, _u8p, _u8p, _i3, ctypes.c_double],
            "or_amr_restrict": [_dp, _dp, _u8p, _i3],
            "or_amr_flag_cells": [_dp, _u8p, _i3, ctypes.c_double, _u8p],
            "or_amr_patch_flags": [_u8p, _u8p, _i3, ctypes.c_int, _u8p],
            "or_amr_prolong_patches": [_dp, _u8p, _i3, _dp],
            "or_step_periodic_fx": [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, _dp],
            "or_step_dual_fx": [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp],
            "or_amr_fill_ghost_s": [_dp, _u8p, _i3, _dp, _dp, _dp, _dp, ctypes.c_double],
            "or_amr_cf_fine_accumulate_s": [_dp, _dp, _u8p, _u8p, _i3, ctypes.c_double],
            "or_amr_cf_coarse_store_s": [_dp, _dp, _u8p, _u8p, _i3, ctypes.c_double],
            "or_amr_fixup_s": [_dp, _dp, _dp, _u8p, _u8p, _i3, ctypes.c_double],
            "or_amr_restrict_s": [_dp, _dp, _u8p, _i3],
            "or_amr_prolong_patches_s": [_dp, _u8p, _i3, _dp, _dp],
        }.items():
            fn = getattr(L, name)
            fn.argtypes = args
        L.or_step_periodic_fx.restype = ctypes.c_int64
        L.or_step_dual_fx.restype = ctypes.c_int64
        _amr = L
    return _amr


def _u8(a):
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u8p)


def _dims(N):
    return _i3(int(N[0]), int(N[1]), int(N[2]))


def covered(mask_f, Nf):
    """Coarse cells covered by the fine level's patches, [Nc_z][Nc_y][Nc_x]."""
    Nc = [n // 2 for n in Nf]
    out = np.empty((Nc[2], Nc[1], Nc[0]), np.uint8)
    amr_lib().or_amr_covered(_u8(mask_f), _dims(Nf), _u8(out))
    return out


def cell_mask(mask):
    """Expand a patch mask to a cell mask (8^3 cells per patch)."""
    return np.repeat(np.repeat(np.repeat(mask.astype(bool), 8, 0), 8, 1), 8, 2)


class Level:
    def __init__(self, N, dual=False):
        self.N = list(N)  # cells per dimension (x, y, z)
        self.mask = np.zeros((N[2] // 8, N[1] // 8, N[0] // 8), np.uint8)
        self.U = np.zeros((5, N[2], N[1], N[0]))
        self.U_prev = self.U.copy()
        self.t = 0.0
        self.t_prev = 0.0
        self.acc = np.zeros((3, 5, N[2], N[1], N[0]))   # fine-flux sums on this (coarse) level's faces
        self.cfl = np.zeros((3, 5, N[2], N[1], N[0]))   # dt_c * F_c on this level's coarse-fine faces
        self.dt_prev = None
        if dual:  # the entropy per unit volume and its flux registers
            self.S = np.ones((N[2], N[1], N[0]))
            self.S_prev = self.S.copy()
            self.acc_s = np.zeros((3, N[2], N[1], N[0]))
            self.cfl_s = np.zeros((3, N[2], N[1], N[0]))

    @property
    def empty(self):
        return not self.mask.any()


class OracleHierarchy:
    def __init__(self, U_root, lmax, gamma, cfl, theta, nbuf, c_inc=0.1, c_dec=0.1, box=1.0,
                 regrid_at_start=True, S_root=None, dual_xi=1e-2, shared_dt=False):
        _, nz, ny, nx = U_root.shape
        self.root_n = (nx, ny, nz)
        self.lmax, self.gamma, self.cfl_c, self.theta = lmax, gamma, cfl, theta
        self.nbuf = list(nbuf)
        self.c_inc, self.c_dec, self.box = c_inc, c_dec, box
        # shared time-step integration (section 2.6): one dt for every level,
        # the minimum of the levels' constraints
        self.shared_dt = shared_dt
        self._shared_step = None
        self.dual = S_root is not None
        self.dual_xi = dual_xi
        self.lv = [Level([n << l for n in self.root_n], self.dual) for l in range(lmax + 1)]
        L0 = self.lv[0]
        L0.mask[:] = 1
        L0.U = np.ascontiguousarray(U_root, dtype=np.float64).copy()
        L0.U_prev = L0.U.copy()
        if self.dual:
            L0.S = np.ascontiguousarray(S_root, dtype=np.float64).copy()
            L0.S_prev = L0.S.copy()
        self.n_updates = 0
        self.log = []  # (level, dt) of every level step, in order
        if regrid_at_start:
            for l in range(lmax):
                self.regrid(l)

    # ---- helpers ------------------------------------------------------------------

    def dh(self, l):
        return self.box / self.root_n[0] / (1 << l)

    def present(self, l):
        return cell_mask(self.lv[l].mask)

    def leaf(self, l):
        p = self.present(l)
        if l < self.lmax and not self.lv[l + 1].empty:
            cov = covered(self.lv[l + 1].mask, self.lv[l + 1].N).astype(bool)
            p &= ~cov
        return p

    def fill_ghost(self, l, t):
        """Section 3.2: ghosts of level l at time t from level l-1."""
        if l == 0:
            return
        c, f = self.lv[l - 1], self.lv[l]
        if c.t == c.t_prev or t == c.t:
            w = 1.0
        else:
            w = (t - c.t_prev) / (c.t - c.t_prev)
        amr_lib().or_amr_fill_ghost(_ptr(f.U), _u8(f.mask), _dims(f.N), _ptr(c.U_prev), _ptr(c.U), w)
        if self.dual:
            amr_lib().or_amr_fill_ghost_s(_ptr(f.S), _u8(f.mask), _dims(f.N), _ptr(c.S_prev), _ptr(c.S),
                                          _ptr(c.U_prev), _ptr(c.U), w)

    def min_dt(self, l):
        """The scheme's CFL condition (Eq. CFL2, CFL1 for CTU) over the cells of
        the level's patches."""
        from . import scheme_max_speed
        cells = self.lv[l].U[:, self.present(l)]
        s = scheme_max_speed(np.ascontiguousarray(cells).reshape(5, -1, 1, 1), self.gamma)
        if not s > 0:
            raise FloatingPointError("unphysical state")
        return self.cfl_c * self.dh(l) / s

    def advance_level(self, l, dt):
        """One MUSCL-Hancock step of every patch of level l, with flux registers."""
        L = self.lv[l]
        self.fill_ghost(l, L.t)
        N = L.N
        Un = np.empty_like(L.U)
        FX = np.empty((3, 5, N[2], N[1], N[0]))
        if self.dual:
            Sn = np.empty_like(L.S)
            FXs = np.empty((3, N[2], N[1], N[0]))
            nb = amr_lib().or_step_dual_fx(_ptr(L.U), _ptr(L.S), _ptr(Un), _ptr(Sn), N[0], N[1], N[2], self.dh(l),
                                           dt, self.gamma, self.dual_xi, _ptr(FX), _ptr(FXs))
            if nb < 0:
                raise ValueError("dual energy is built for MUSCL-Hancock only")
        else:
            amr_lib().or_step_periodic_fx(_ptr(L.U), _ptr(Un), N[0], N[1], N[2], self.dh(l), dt, self.gamma,
                                          _ptr(FX))
        pres = self.present(l)
        new = L.U.copy()
        new[:, pres] = Un[:, pres]
        if self.dual:
            news = L.S.copy()
            news[pres] = Sn[pres]
            L.S_prev, L.S = L.S, news
        rho = new[0][pres]
        v2 = (new[1][pres] ** 2 + new[2][pres] ** 2 + new[3][pres] ** 2) / rho
        if not ((rho > 0).all() and (new[4][pres] - 0.5 * v2 > 0).all()):
            raise FloatingPointError(f"unphysical cells on level {l}")
        L.U_prev, L.U = L.U, new
        L.t_prev = L.t
        self.n_updates += int(pres.sum())
        self.log.append((l, dt))
        if l > 0:
            c = self.lv[l - 1]
            cov = covered(L.mask, N)
            amr_lib().or_amr_cf_fine_accumulate(_ptr(c.acc), _ptr(FX), _u8(cov), _u8(c.mask), _dims(c.N), dt)
            if self.dual:
                amr_lib().or_amr_cf_fine_accumulate_s(_ptr(c.acc_s), _ptr(FXs), _u8(cov), _u8(c.mask), _dims(c.N),
                                                      dt)
        if l < self.lmax and not self.lv[l + 1].empty:
            cov = covered(self.lv[l + 1].mask, self.lv[l + 1].N)
            amr_lib().or_amr_cf_coarse_store(_ptr(L.cfl), _ptr(FX), _u8(cov), _u8(L.mask), _dims(N), dt)
            L.acc[:] = 0.0
            if self.dual:
                amr_lib().or_amr_cf_coarse_store_s(_ptr(L.cfl_s), _ptr(FXs), _u8(cov), _u8(L.mask), _dims(N), dt)
                L.acc_s[:] = 0.0

    def flux_fixup(self, l):
        """Section 2.2 synchronisation of level l with level l+1."""
        c, f = self.lv[l], self.lv[l + 1]
        cov = covered(f.mask, f.N)
        amr_lib().or_amr_fixup(_ptr(c.U), _ptr(c.acc), _ptr(c.cfl), _u8(cov), _u8(c.mask), _dims(c.N), self.dh(l))
        amr_lib().or_amr_restrict(_ptr(c.U), _ptr(f.U), _u8(cov), _dims(c.N))
        if self.dual:
            amr_lib().or_amr_fixup_s(_ptr(c.S), _ptr(c.acc_s), _ptr(c.cfl_s), _u8(cov), _u8(c.mask), _dims(c.N),
                                     self.dh(l))
            amr_lib().or_amr_restrict_s(_ptr(c.S), _ptr(f.S), _u8(cov), _dims(c.N))

    # ---- W-cycle (section 2.1 pseudo-code) -------------------------------------------

    def advance(self, l, dt0=None):
        L = self.lv[l]
        if l == 0:
            if self.shared_dt:
                # the time-step constraint evaluated on all levels, the minimum taken
                if dt0 is None:
                    dt = min(self.min_dt(k) for k in range(self.lmax + 1) if not self.lv[k].empty)
                else:
                    dt = dt0
                self._shared_step = dt
            else:
                dt = self.min_dt(0) if dt0 is None else dt0
                dt = self._dec_rule(l, dt)
            target = L.t + dt
        else:
            target = self.lv[l - 1].t
        while L.t < target:
            last = False
            if l == 0:
                step = dt  # the root level takes one step of exactly dt per call
            else:
                # shared: the root's dt, which lands on the parent's time in one step
                step = self._shared_step if self.shared_dt else self.min_dt(l)
                if (1.0 + self.c_inc) * step > target - L.t:
                    step = target - L.t
                    last = True
                elif not self.shared_dt:
                    step = self._dec_rule(l, step)
            self.advance_level(l, step)
            L.t = target if (last or l == 0) else L.t + step
            L.dt_prev = step
            if l < self.lmax and not self.lv[l + 1].empty:
                self.advance(l + 1)
                self.flux_fixup(l)
            if l < self.lmax:
                self.regrid(l)

    def _dec_rule(self, l, dt):
        if l < self.lmax and self.lv[l + 1].dt_prev is not None and not self.lv[l + 1].empty:
            d2 = 2.0 * self.lv[l + 1].dt_prev
            if dt > d2 and (1.0 - self.c_dec) * dt < d2:
                return d2
        return dt

    # ---- regrid (section 2.1) --------------------------------------------------------

    def cell_flags(self, l):
        L = self.lv[l]
        self.fill_ghost(l, L.t)
        cf = np.empty((L.N[2], L.N[1], L.N[0]), np.uint8)
        amr_lib().or_amr_flag_cells(_ptr(L.U), _u8(L.mask), _dims(L.N), self.theta, _u8(cf))
        return cf

    def patch_flags(self, l, cell_flags=None):
        L = self.lv[l]
        cf = self.cell_flags(l) if cell_flags is None else \
            np.ascontiguousarray((cell_flags.astype(bool) & cell_mask(L.mask)).astype(np.uint8))
        pf = np.empty_like(L.mask)
        amr_lib().or_amr_patch_flags(_u8(cf), _u8(L.mask), _dims(L.N), self.nbuf[l], _u8(pf))
        return pf

    def regrid(self, l, cell_flags=None):
        """Rebuild level l+1 from the flags of level l at the level's time
        (cell_flags: optional hand-made cell flags of level l, for tests)."""
        L, F = self.lv[l], self.lv[l + 1]
        flags = self.patch_flags(l, cell_flags).astype(bool)
        present = L.mask.astype(bool)
        refined = self._refined(l)
        keep = np.zeros_like(present)
        if l + 2 <= self.lmax and not self.lv[l + 2].empty:
            # fine patches with children, and the 26 neighbour positions of each
            fine_ref = self._refined(l + 1)
            pos = np.argwhere(fine_ref)
            P = np.array(present.shape)
            for q in pos:
                for d in np.ndindex(3, 3, 3):
                    keep[tuple(((q + np.array(d) - 1) // 2) % P)] = True
        nest_ok = np.ones_like(present)
        if l > 0:
            for d in np.ndindex(3, 3, 3):
                if d == (1, 1, 1):
                    continue
                nest_ok &= np.roll(present, shift=tuple(1 - np.array(d)), axis=(0, 1, 2))
        new_ref = present & ((flags & nest_ok) | (keep & refined))
        newmask = np.repeat(np.repeat(np.repeat(new_ref, 2, 0), 2, 1), 2, 2).astype(np.uint8)
        created = newmask.astype(bool) & ~F.mask.astype(bool)
        Unew = F.U.copy()
        if created.any():
            amr_lib().or_amr_prolong_patches(_ptr(Unew), _u8(created.astype(np.uint8)), _dims(F.N), _ptr(L.U))
        F.U = Unew
        F.mask = newmask
        F.U_prev = F.U.copy()
        if self.dual:
            Snew = F.S.copy()
            if created.any():
                amr_lib().or_amr_prolong_patches_s(_ptr(Snew), _u8(created.astype(np.uint8)), _dims(F.N),
                                                   _ptr(L.S), _ptr(L.U))
            F.S = Snew
            F.S_prev = F.S.copy()
        F.t = F.t_prev = L.t
        if F.empty:
            F.dt_prev = None

    def _refined(self, l):
        """Patches of level l that have children on level l+1."""
        F = self.lv[l + 1]
        m = F.mask.astype(bool)
        return m[0::2, 0::2, 0::2] & self.lv[l].mask.astype(bool)

    # ---- diagnostics ----------------------------------------------------------------

    def conserved_total(self):
        tot = np.zeros(5)
        for l in range(self.lmax + 1):
            if self.lv[l].empty:
                continue
            lf = self.leaf(l)
            dV = self.dh(l) ** 3
            for v in range(5):
                tot[v] += self.lv[l].U[v][lf].sum() * dV
        return tot

    def patch_corners(self, l):
        """Sorted (z, y, x)-ordered list of patch corners (cell units) of level l."""
        pos = np.argwhere(self.lv[l].mask.astype(bool))  # (pz, py, px) rows, lexicographic
        return [(int(p[2]) * 8, int(p[1]) * 8, int(p[0]) * 8) for p in pos]
