"""Oracle discrete adjoint (test infrastructure): reverse-mode tape and
forward-mode tangent of the unchanged oracle step (adjoint_oracle.cpp), and
the adjoint of a run of steps with its time steps frozen."""
import ctypes

import numpy as np

from . import _build, lib as _lib, step_periodic

_ad = None


def ad_lib():
    global _ad
    if _ad is None:
        _lib()  # builds everything
        L = ctypes.CDLL(_build.ADLIB)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.or_adj_step.argtypes = [vp, vp, vp, i, i, i, d, d, d]
        L.or_jvp_step.argtypes = [vp, vp, vp, i, i, i, d, d, d]
        L.or_adj_hllc.argtypes = [vp, vp, i, d, vp, vp, vp]
        _ad = L
    return _ad


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def adj_step(U, lam_np1, dh, dt, gamma):
    """(dS/dU)^T lam_np1 for one periodic step S (dt fixed)."""
    U, lam = _c(U), _c(lam_np1)
    out = np.empty_like(U)
    _, nz, ny, nx = U.shape
    ad_lib().or_adj_step(U.ctypes.data, lam.ctypes.data, out.ctypes.data, nx, ny, nz, dh, dt, gamma)
    return out


def jvp_step(U, V, dh, dt, gamma):
    """(dS/dU) V for one periodic step S (dt fixed)."""
    U, V = _c(U), _c(V)
    out = np.empty_like(U)
    _, nz, ny, nx = U.shape
    ad_lib().or_jvp_step(U.ctypes.data, V.ctypes.data, out.ctypes.data, nx, ny, nz, dh, dt, gamma)
    return out


def adj_hllc(UL, UR, d, gamma, lamF):
    """(dF/dUL)^T lamF, (dF/dUR)^T lamF of one HLLC face evaluation."""
    UL, UR, lamF = _c(UL), _c(UR), _c(lamF)
    a, b = np.empty(5), np.empty(5)
    ad_lib().or_adj_hllc(UL.ctypes.data, UR.ctypes.data, d, gamma, lamF.ctypes.data, a.ctypes.data, b.ctypes.data)
    return a, b


def run_frozen(U0, dts, dh, gamma):
    """Forward run with a given dt sequence; returns all states."""
    states = [_c(U0)]
    for dt in dts:
        U, _ = step_periodic(states[-1], dh, dt, gamma)
        states.append(U)
    return states


def loss(U, rho_target, dV):
    """L = 1/2 sum_cells (rho - rho*)^2 dV."""
    return 0.5 * float(((U[0] - rho_target) ** 2).sum()) * dV


def gradient(U0, dts, dh, gamma, rho_target):
    """dL/dU0 of L(U_N) by the reverse sweep over the frozen dt sequence."""
    dV = dh ** 3
    states = run_frozen(U0, dts, dh, gamma)
    lam = np.zeros_like(states[-1])
    lam[0] = (states[-1][0] - rho_target) * dV
    for k in range(len(dts) - 1, -1, -1):
        lam = adj_step(states[k], lam, dh, dts[k], gamma)
    return lam, states
