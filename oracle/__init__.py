"""FP64 CPU oracle for the GAMER-2 patch-group hydro update (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path:
the C sources here are compiled by ``oracle/build.py`` into ``liboracle.so``
and called through ctypes on numpy arrays in the dense whole-level layout
``U[var][z][y][x]``.

Every function cites the paper passage it follows (GAMER-2, Schive et al.
2018): section 2.2 (Hydrodynamics: MUSCL-Hancock, PLM, van Leer-type limiter,
HLLC; restriction and flux fix-up), section 2.6 (Eq. CFL2), section 2.1 (AMR
structure, adaptive time-step pseudo-code, refinement and flag buffers).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        L = _lib
        L.or_prim.argtypes = [_dp, _dp, ctypes.c_double]
        L.or_cons.argtypes = [_dp, _dp, ctypes.c_double]
        L.or_flux.argtypes = [_dp, ctypes.c_int, ctypes.c_double, _dp]
        L.or_vanleer.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_vanleer.restype = ctypes.c_double
        L.or_hllc.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double, _dp]
        L.or_hlle.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double, _dp]
        L.or_roe.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double, _dp]
        L.or_exact_flux.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_double, _dp]
        L.or_set_scheme.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.or_set_vl.argtypes = [ctypes.c_int]
        L.or_set_ctu.argtypes = [ctypes.c_int]
        L.or_set_ppm.argtypes = [ctypes.c_int]
        L.or_set_fallback.argtypes = [ctypes.c_int]
        L.or_fallback_counts.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        L.or_step_dual.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_step_dual.restype = ctypes.c_int64
        L.or_step_gravity_predictor.argtypes = [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_step_gravity_predictor.restype = ctypes.c_int64
        L.or_ppm_faces.argtypes = [_dp, _dp, _dp]
        L.or_max_speed1.argtypes = [_dp, ctypes.c_int64, ctypes.c_double]
        L.or_max_speed1.restype = ctypes.c_double
        L.or_dt_cfl1.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_dt_cfl1.restype = ctypes.c_double
        for name in ("or_gminmod", "or_vl_gminmod"):
            getattr(L, name).argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            getattr(L, name).restype = ctypes.c_double
        for name in ("or_albada", "or_slope"):
            getattr(L, name).argtypes = [ctypes.c_double, ctypes.c_double]
            getattr(L, name).restype = ctypes.c_double
        L.or_max_speed.argtypes = [_dp, ctypes.c_int64, ctypes.c_double]
        L.or_max_speed.restype = ctypes.c_double
        L.or_dt_cfl2.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_dt_cfl2.restype = ctypes.c_double
        L.or_step_periodic.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_step_periodic.restype = ctypes.c_int64
        L.or_conserved_sum.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, _dp]
        L.or_exact_star.argtypes = [ctypes.c_double] * 7 + [_dp, _dp]
        L.or_exact_pstar_bisect.argtypes = [ctypes.c_double] * 7
        L.or_exact_pstar_bisect.restype = ctypes.c_double
        L.or_exact_sample.argtypes = [ctypes.c_double] * 7 + [_dp, ctypes.c_int, _dp, _dp, _dp]
        for extra in ("_register_amr", "_register_adjoint"):
            fn = globals().get(extra)
            if fn is not None:
                fn(L)
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


# ---- pointwise pieces (section 2.2) -----------------------------------------

def prim(U, gamma):
    """Conserved -> primitive for one state (ideal gas)."""
    U = _vec(U)
    W = np.empty(5)
    lib().or_prim(_ptr(U), _ptr(W), gamma)
    return W


def cons(W, gamma):
    """Primitive -> conserved for one state."""
    W = _vec(W)
    U = np.empty(5)
    lib().or_cons(_ptr(W), _ptr(U), gamma)
    return U


def flux(U, d, gamma):
    """Physical Euler flux along direction d of one conserved state."""
    U = _vec(U)
    F = np.empty(5)
    lib().or_flux(_ptr(U), d, gamma, _ptr(F))
    return F


def vanleer(a, b):
    """van Leer-type limiter, 2ab/(a+b) when ab>0 else 0 (section 2.2)."""
    return lib().or_vanleer(a, b)


# ---- scheme options (section 2.2 lists the limiters and Riemann solvers) -----

LIM_VANLEER, LIM_GMINMOD, LIM_ALBADA, LIM_VL_GMINMOD = 0, 1, 2, 3
RS_HLLC, RS_HLLE, RS_ROE, RS_EXACT = 0, 1, 2, 3


_ctu = [False]  # the CTU scheme takes its dt from Eq. CFL1


def set_scheme(limiter=LIM_VANLEER, riemann=RS_HLLC, theta=1.5, vl=False, ctu=False, ppm=False, fallback=False):
    """Select the slope limiter, the Riemann solver, the generalized minmod
    coefficient, the integration scheme (VL half step, CTU, else
    MUSCL-Hancock), PPM reconstruction (else PLM) and the per-cell remedies
    for unphysical results of every later oracle step (process-wide)."""
    assert not (vl and ctu)
    lib().or_set_scheme(limiter, riemann, theta)
    lib().or_set_vl(1 if vl else 0)
    lib().or_set_ctu(1 if ctu else 0)
    lib().or_set_ppm(1 if ppm else 0)
    lib().or_set_fallback(1 if fallback else 0)
    _ctu[0] = bool(ctu)


class scheme:
    """Context manager: a scheme for the steps inside, the default after."""

    def __init__(self, limiter=LIM_VANLEER, riemann=RS_HLLC, theta=1.5, vl=False, ctu=False, ppm=False,
                 fallback=False):
        self.args = (limiter, riemann, theta, vl, ctu, ppm, fallback)

    def __enter__(self):
        set_scheme(*self.args)
        return self

    def __exit__(self, *exc):
        set_scheme()
        return False


def gminmod(a, b, theta):
    """Generalized minmod slope: sign(a) min(theta|a|, |a+b|/2, theta|b|) if ab>0."""
    return lib().or_gminmod(a, b, theta)


def albada(a, b):
    """van Albada-type slope: ab(a+b)/(a^2+b^2) if ab>0."""
    return lib().or_albada(a, b)


def vl_gminmod(a, b, theta):
    """Hybrid slope: the smaller of the van Leer-type and generalized minmod."""
    return lib().or_vl_gminmod(a, b, theta)


def slope(a, b):
    """The slope of the selected limiter."""
    return lib().or_slope(a, b)


def ppm_faces(w5):
    """PPM face values (W_L, W_R) of the middle cell of five cell values."""
    w5 = np.ascontiguousarray(w5, dtype=np.float64)
    a, b = np.empty(1), np.empty(1)
    lib().or_ppm_faces(_ptr(w5), _ptr(a), _ptr(b))
    return float(a[0]), float(b[0])


def hlle(UL, UR, d, gamma):
    """HLLE flux (Einfeldt 1991) through a face normal to d."""
    UL, UR = _vec(UL), _vec(UR)
    F = np.empty(5)
    lib().or_hlle(_ptr(UL), _ptr(UR), d, gamma, _ptr(F))
    return F


def roe(UL, UR, d, gamma):
    """Roe flux (with the Harten-Hyman entropy fix) through a face normal to d."""
    UL, UR = _vec(UL), _vec(UR)
    F = np.empty(5)
    lib().or_roe(_ptr(UL), _ptr(UR), d, gamma, _ptr(F))
    return F


def exact_flux(UL, UR, d, gamma):
    """Godunov flux of the exact Riemann solution through a face normal to d."""
    UL, UR = _vec(UL), _vec(UR)
    F = np.empty(5)
    lib().or_exact_flux(_ptr(UL), _ptr(UR), d, gamma, _ptr(F))
    return F


def hllc(UL, UR, d, gamma):
    """HLLC flux through a face normal to d (section 2.2, HLLC solver)."""
    UL, UR = _vec(UL), _vec(UR)
    F = np.empty(5)
    lib().or_hllc(_ptr(UL), _ptr(UR), d, gamma, _ptr(F))
    return F


# ---- whole-level operations ---------------------------------------------------

def max_speed(U, gamma):
    """max over cells of |vx|+|vy|+|vz|+3c_s (denominator of Eq. CFL2)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_max_speed(_ptr(U), U[0].size, gamma)


def dt_cfl2(U, gamma, cfl, dh):
    """Eq. CFL2: dt = C_CFL dh / max(|vx|+|vy|+|vz|+3c_s)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_dt_cfl2(_ptr(U), U[0].size, gamma, cfl, dh)


def max_speed1(U, gamma):
    """max over cells of max(|vx|,|vy|,|vz|)+c_s (denominator of Eq. CFL1)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_max_speed1(_ptr(U), U[0].size, gamma)


def dt_cfl1(U, gamma, cfl, dh):
    """Eq. CFL1: dt = C_CFL dh / max(max(|vx|,|vy|,|vz|)+c_s)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_dt_cfl1(_ptr(U), U[0].size, gamma, cfl, dh)


def scheme_max_speed(U, gamma):
    """The CFL denominator of the selected scheme (CFL1 for CTU, else CFL2)."""
    return max_speed1(U, gamma) if _ctu[0] else max_speed(U, gamma)


def dt_cfl(U, gamma, cfl, dh):
    """The time step of the selected scheme: Eq. CFL1 for CTU, else CFL2."""
    return dt_cfl1(U, gamma, cfl, dh) if _ctu[0] else dt_cfl2(U, gamma, cfl, dh)


def step_periodic(U, dh, dt, gamma):
    """One MUSCL-Hancock + PLM + HLLC step on a periodic uniform grid.

    U: [5][nz][ny][nx] float64.  Returns (U_new, n_unphysical)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    _, nz, ny, nx = U.shape
    Un = np.empty_like(U)
    nbad = lib().or_step_periodic(_ptr(U), _ptr(Un), nx, ny, nz, dh, dt, gamma)
    return Un, nbad


def run_periodic(U, dh, gamma, cfl, n_steps):
    """n_steps steps, each with dt from the scheme's CFL condition (Eq. CFL1
    for CTU, else CFL2) on the state at the step's start.

    Returns (U, list of dt)."""
    dts = []
    for _ in range(n_steps):
        dt = dt_cfl(U, gamma, cfl, dh)
        if not dt > 0:
            raise FloatingPointError("unphysical state (rho<=0 or P<=0)")
        U, nbad = step_periodic(U, dh, dt, gamma)
        if nbad:
            raise FloatingPointError(f"{nbad} unphysical cells")
        dts.append(dt)
    return U, dts


def entropy(U, gamma):
    """The dual-energy variable s = P / rho^(gamma-1) of a state [5][...]."""
    U = np.asarray(U, dtype=np.float64)
    P = (gamma - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
    return P / U[0] ** (gamma - 1.0)


def step_dual(U, S, dh, dt, gamma, xi=1e-2):
    """One MUSCL-Hancock step with the dual-energy formalism (entropy S per
    unit volume carried as a passive scalar; E corrected from S where
    E_the / E_kin < xi, S reset from E elsewhere).  Returns (U, S, nbad)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    nz, ny, nx = U.shape[1:]
    Un, Sn = np.empty_like(U), np.empty_like(S)
    nbad = lib().or_step_dual(_ptr(U), _ptr(S), _ptr(Un), _ptr(Sn), nx, ny, nz, dh, dt, gamma, xi)
    if nbad < 0:
        raise ValueError("dual energy is built for MUSCL-Hancock only")
    return Un, Sn, nbad


def step_gravity_predictor(U, g, dh, dt, gamma):
    """The gravity coupling's predictor: the MUSCL-Hancock (or, with the CTU
    scheme selected, the CTU) step with (dt/2)(0, rho g, m.g) of each
    reconstructed face state added to its predicted state (CTU: after the
    normal predictor, before the transverse correction); g [3][...] the
    acceleration at t^n.  Returns (U*, nbad)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    nz, ny, nx = U.shape[1:]
    Un = np.empty_like(U)
    nbad = lib().or_step_gravity_predictor(_ptr(U), _ptr(g), _ptr(Un), nx, ny, nz, dh, dt, gamma)
    if nbad < 0:
        raise ValueError("the gravity coupling is built for MUSCL-Hancock and CTU")
    return Un, nbad


def fallback_counts(reset=True):
    """Cells the per-cell remedies handled since the last reset: (fixed by the
    first-order unsplit update, fixed by the split one, still unphysical)."""
    out = (ctypes.c_int64 * 3)()
    lib().or_fallback_counts(out, 1 if reset else 0)
    return tuple(out)


def step_retry(U, dh, dt, gamma, dt_min, factor=0.8):
    """One step with the level remedies (iv)-(v): while cells stay unphysical
    after the per-cell remedies, retry from U with dt * factor; give up below
    dt_min.  Returns (U_new, dt taken) or raises FloatingPointError."""
    while True:
        Un, nbad = step_periodic(U, dh, dt, gamma)
        if nbad == 0:
            return Un, dt
        dt *= factor
        if dt < dt_min:
            raise FloatingPointError(f"{nbad} unphysical cells at the minimum dt")


def conserved_sum(U, dV):
    """Sum of U*dV per variable, pairwise in fixed cell order."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty(5)
    lib().or_conserved_sum(_ptr(U), U[0].size, dV, _ptr(out))
    return out


# ---- instrumented operation count ---------------------------------------------

def count_flops(U, gamma):
    """Per-cell FP64 operation counts of one oracle step and of one Eq. CFL2
    signal-speed evaluation on state U (flop_count.cpp): a dict with keys
    add, mul, div, sqrt, cmp for 'step' and 'speed'."""
    lib()
    L = ctypes.CDLL(_build.FLOPLIB)
    U = np.ascontiguousarray(U, dtype=np.float64)
    _, nz, ny, nx = U.shape
    out = np.zeros(12)
    L.or_count_flops(U.ctypes.data_as(ctypes.c_void_p), nx, ny, nz, ctypes.c_double(gamma),
                     out.ctypes.data_as(ctypes.c_void_p))
    keys = ("add", "mul", "div", "sqrt", "cmp", "other")
    return {"step": dict(zip(keys, out[:6])), "speed": dict(zip(keys, out[6:]))}


# ---- exact Riemann solver (validation only) ----------------------------------

def exact_star(rl, ul, pl, rr, ur, pr, gamma):
    ps, us = ctypes.c_double(), ctypes.c_double()
    lib().or_exact_star(rl, ul, pl, rr, ur, pr, gamma, ctypes.byref(ps), ctypes.byref(us))
    return ps.value, us.value


def exact_pstar_bisect(rl, ul, pl, rr, ur, pr, gamma):
    return lib().or_exact_pstar_bisect(rl, ul, pl, rr, ur, pr, gamma)


def exact_sample(left, right, gamma, xi):
    xi = _vec(xi)
    n = xi.size
    r, u, p = np.empty(n), np.empty(n), np.empty(n)
    lib().or_exact_sample(*left, *right, gamma, _ptr(xi), n, _ptr(r), _ptr(u), _ptr(p))
    return r, u, p
