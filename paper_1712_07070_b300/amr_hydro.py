"""Thin ctypes binding of the C ABI in include/amr_hydro.h (same names).

Argument marshalling only: every step of the hydro path runs in the CUDA
library ``libamr_hydro.so``.  Loading fails loudly if the library is missing;
there is no CPU fallback.  Device arrays are passed as raw pointers, e.g.
``tensor.data_ptr()`` of a CUDA torch tensor.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libamr_hydro.so")

AMR_OK, AMR_E_INVAL, AMR_E_NOMEM, AMR_E_CUDA, AMR_E_UNPHYSICAL, AMR_E_TIMEOUT, AMR_E_NESTING = range(7)
AMR_FP64, AMR_FP32_ACC64 = 0, 1
AMR_LIM_VANLEER, AMR_LIM_GMINMOD, AMR_LIM_ALBADA, AMR_LIM_VL_GMINMOD = 0, 1, 2, 3
AMR_RS_HLLC, AMR_RS_HLLE, AMR_RS_ROE, AMR_RS_EXACT = 0, 1, 2, 3
AMR_SCHEME_MH, AMR_SCHEME_VL, AMR_SCHEME_CTU = 0, 1, 2
AMR_RECON_PLM, AMR_RECON_PPM = 0, 1
AMR_GRAVITY_PERIODIC, AMR_GRAVITY_ISOLATED = 0, 1

# every symbol include/amr_hydro.h declares
SYMBOLS = (
    "amr_hydro_init", "amr_hydro_destroy", "amr_hydro_set_level", "amr_hydro_get_state",
    "amr_hydro_touch_level",
    "amr_hydro_fill_ghost", "amr_hydro_advance_level", "amr_hydro_flux_fixup", "amr_hydro_min_dt",
    "amr_hydro_regrid_flags", "amr_hydro_conserved_sum", "amr_hydro_set_box",
    "amr_hydro_advance_boxes", "amr_hydro_box_state", "amr_hydro_step_adjoint",
    "amr_hydro_strerror", "amr_hydro_uniform_tables", "amr_hydro_pack_uniform",
    "amr_hydro_unpack_uniform", "amr_hydro_step_uniform_noalloc", "amr_hydro_bind_level",
    "amr_hydro_regrid", "amr_hydro_advance_root", "amr_hydro_level_info", "amr_hydro_box_tuning",
    "amr_hydro_advance_host", "amr_hydro_set_entropy", "amr_hydro_poisson_root", "amr_hydro_poisson_level",
    "amr_hydro_advance_gravity", "amr_hydro_poisson_level_t", "amr_hydro_phase_timing", "amr_hydro_phase_times",
    "amr_hydro_set_box_entropy", "amr_hydro_set_gravity", "amr_hydro_level_gravity", "amr_hydro_set_shared_dt",
)
AMR_PH_GHOST, AMR_PH_STEP, AMR_PH_FIXUP, AMR_PH_REGRID, AMR_PH_DT = range(5)
AMR_N_PHASES = 5
PHASE_NAMES = ("ghost fill", "step", "fix-up", "regrid", "dt")


class amr_hydro_params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("c_inc", ctypes.c_double),
        ("c_dec", ctypes.c_double), ("theta", ctypes.c_double), ("lmax", ctypes.c_int),
        ("nbuf", ctypes.c_int * 8), ("prec", ctypes.c_int), ("periodic", ctypes.c_int * 3),
        ("box", ctypes.c_double * 3), ("root_n", ctypes.c_int * 3), ("max_patches", ctypes.c_int),
        ("limiter", ctypes.c_int), ("riemann", ctypes.c_int), ("minmod_coeff", ctypes.c_double),
        ("scheme", ctypes.c_int), ("recon", ctypes.c_int), ("fallback", ctypes.c_int), ("dt_min", ctypes.c_double),
        ("dual_energy", ctypes.c_int), ("dual_xi", ctypes.c_double), ("gravity_bc", ctypes.c_int),
    ]


class AmrHydroError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


_lib = None
_vp, _dp, _ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    """Load libamr_hydro.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run python -m paper_1712_07070_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "amr_hydro_init": [ctypes.POINTER(amr_hydro_params), _vp, ctypes.POINTER(_vp)],
        "amr_hydro_destroy": [_vp],
        "amr_hydro_set_level": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_double],
        "amr_hydro_get_state": [_vp, ctypes.c_int, _ip, _dp, _dp],
        "amr_hydro_touch_level": [_vp, ctypes.c_int],
        "amr_hydro_set_entropy": [_vp, ctypes.c_int, _vp, _vp],
        "amr_hydro_poisson_root": [_vp, ctypes.c_double, _vp, _vp, ctypes.c_int],
        "amr_hydro_poisson_level_t": [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp, _vp,
                                      ctypes.c_double, _vp, _vp, ctypes.c_int],
        "amr_hydro_advance_gravity": [_vp, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, ctypes.c_int,
                                      ctypes.c_double],
        "amr_hydro_poisson_level": [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp, _vp,
                                    _vp, ctypes.c_int],
        "amr_hydro_fill_ghost": [_vp, ctypes.c_int, ctypes.c_double],
        "amr_hydro_advance_level": [_vp, ctypes.c_int, ctypes.c_double, _i64p],
        "amr_hydro_advance_host": [_vp, _vp, _vp, ctypes.c_double, _dp],
        "amr_hydro_flux_fixup": [_vp, ctypes.c_int],
        "amr_hydro_min_dt": [_vp, ctypes.c_int, _vp],
        "amr_hydro_regrid_flags": [_vp, ctypes.c_int, _vp],
        "amr_hydro_conserved_sum": [_vp, ctypes.c_int, _dp],
        "amr_hydro_set_box": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp],
        "amr_hydro_set_box_entropy": [_vp, ctypes.c_int, _vp, _vp],
        "amr_hydro_set_gravity": [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int],
        "amr_hydro_level_gravity": [_vp, ctypes.c_int, _vp, _vp],
        "amr_hydro_set_shared_dt": [_vp, ctypes.c_int],
        "amr_hydro_advance_boxes": [_vp, ctypes.c_int, _ip, ctypes.c_int, _vp],
        "amr_hydro_box_state": [_vp, ctypes.c_int, _ip],
        "amr_hydro_step_adjoint": [_vp, ctypes.c_int, ctypes.c_double, _vp, _vp, _vp],
        "amr_hydro_strerror": [ctypes.c_int],
        "amr_hydro_uniform_tables": [_ip, _vp, _vp, _vp, _vp],
        "amr_hydro_pack_uniform": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp],
        "amr_hydro_unpack_uniform": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp],
        "amr_hydro_box_tuning": [_vp, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_float)],
        "amr_hydro_bind_level": [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp],
        "amr_hydro_regrid": [_vp, ctypes.c_int],
        "amr_hydro_advance_root": [_vp, ctypes.c_double, _i64p],
        "amr_hydro_level_info": [_vp, ctypes.c_int, _ip, _ip],
        "amr_hydro_phase_timing": [_vp, ctypes.c_int],
        "amr_hydro_phase_times": [_vp, _dp, _i64p],
        "amr_hydro_step_uniform_noalloc": [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           _vp, _vp, _vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.amr_hydro_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def strerror(status):
    return lib().amr_hydro_strerror(status).decode()


def check(status, where):
    if status != AMR_OK:
        raise AmrHydroError(status, where)
    return status


def _p(x):
    """Raw pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# ---- same-name wrappers -----------------------------------------------------------

def amr_hydro_init(params, stream=None):
    ctx = _vp()
    check(lib().amr_hydro_init(ctypes.byref(params), _p(stream), ctypes.byref(ctx)), "amr_hydro_init")
    return ctx


def amr_hydro_destroy(ctx):
    check(lib().amr_hydro_destroy(ctx), "amr_hydro_destroy")


def amr_hydro_set_level(ctx, level, n_patches, U_a, U_b, corner, sib, parent=None, child_group=None, t=0.0):
    check(lib().amr_hydro_set_level(ctx, level, n_patches, _p(U_a), _p(U_b), _p(corner), _p(sib),
                                    _p(parent), _p(child_group), t), "amr_hydro_set_level")


def amr_hydro_get_state(ctx, level):
    cur, tc, tp = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    check(lib().amr_hydro_get_state(ctx, level, ctypes.byref(cur), ctypes.byref(tc), ctypes.byref(tp)),
          "amr_hydro_get_state")
    return cur.value, tc.value, tp.value


def amr_hydro_touch_level(ctx, level):
    check(lib().amr_hydro_touch_level(ctx, level), "amr_hydro_touch_level")


def amr_hydro_fill_ghost(ctx, level, t):
    check(lib().amr_hydro_fill_ghost(ctx, level, t), "amr_hydro_fill_ghost")


def amr_hydro_advance_level(ctx, level, dt, count_unphysical=False):
    """Returns the unphysical-cell count when count_unphysical (synchronises)."""
    if count_unphysical:
        n = ctypes.c_int64()
        st = lib().amr_hydro_advance_level(ctx, level, dt, ctypes.byref(n))
        if st not in (AMR_OK, AMR_E_UNPHYSICAL):
            check(st, "amr_hydro_advance_level")
        return n.value
    check(lib().amr_hydro_advance_level(ctx, level, dt, None), "amr_hydro_advance_level")
    return None


def amr_hydro_set_entropy(ctx, level, S_a, S_b):
    check(lib().amr_hydro_set_entropy(ctx, level, _p(S_a), _p(S_b)), "amr_hydro_set_entropy")


def amr_hydro_poisson_root(ctx, G, phi, acc=None, acc_order=2):
    check(lib().amr_hydro_poisson_root(ctx, G, _p(phi), _p(acc), acc_order), "amr_hydro_poisson_root")


def amr_hydro_advance_gravity(ctx, dt, G, acc_n, phi_new, acc_new, acc_order=2, c_acc=0.0):
    check(lib().amr_hydro_advance_gravity(ctx, dt, G, _p(acc_n), _p(phi_new), _p(acc_new), acc_order, c_acc),
          "amr_hydro_advance_gravity")


def amr_hydro_poisson_level_t(ctx, level, G, omega, iters, phi_coarse_old, phi_coarse_new, w, phi, acc=None,
                              acc_order=2):
    check(lib().amr_hydro_poisson_level_t(ctx, level, G, omega, iters, _p(phi_coarse_old), _p(phi_coarse_new), w,
                                          _p(phi), _p(acc), acc_order), "amr_hydro_poisson_level_t")


def amr_hydro_poisson_level(ctx, level, G, omega, iters, phi_coarse, phi, acc=None, acc_order=2):
    check(lib().amr_hydro_poisson_level(ctx, level, G, omega, iters, _p(phi_coarse), _p(phi), _p(acc), acc_order),
          "amr_hydro_poisson_level")


def amr_hydro_flux_fixup(ctx, coarse_level):
    check(lib().amr_hydro_flux_fixup(ctx, coarse_level), "amr_hydro_flux_fixup")


def amr_hydro_min_dt(ctx, level, dt_out=None):
    """Host dt (float) when dt_out is None, else writes the device tensor dt_out."""
    if dt_out is None:
        d = ctypes.c_double()
        check(lib().amr_hydro_min_dt(ctx, level, ctypes.cast(ctypes.byref(d), _vp)), "amr_hydro_min_dt")
        return d.value
    check(lib().amr_hydro_min_dt(ctx, level, _p(dt_out)), "amr_hydro_min_dt")
    return None


def amr_hydro_regrid_flags(ctx, level, patch_flags_dev):
    check(lib().amr_hydro_regrid_flags(ctx, level, _p(patch_flags_dev)), "amr_hydro_regrid_flags")


def amr_hydro_conserved_sum(ctx, level):
    out = (ctypes.c_double * 5)()
    check(lib().amr_hydro_conserved_sum(ctx, level, out), "amr_hydro_conserved_sum")
    return list(out)


def amr_hydro_set_box(ctx, box_id, n, U_a, U_b):
    check(lib().amr_hydro_set_box(ctx, box_id, n, _p(U_a), _p(U_b)), "amr_hydro_set_box")


def amr_hydro_advance_boxes(ctx, box_ids, n_steps, dt_log=None):
    ids = (ctypes.c_int * len(box_ids))(*box_ids)
    check(lib().amr_hydro_advance_boxes(ctx, len(box_ids), ids, n_steps, _p(dt_log)),
          "amr_hydro_advance_boxes")


def amr_hydro_box_state(ctx, box_id):
    cur = ctypes.c_int()
    check(lib().amr_hydro_box_state(ctx, box_id, ctypes.byref(cur)), "amr_hydro_box_state")
    return cur.value


def amr_hydro_box_tuning(ctx):
    g, c, i, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    check(lib().amr_hydro_box_tuning(ctx, ctypes.byref(g), ctypes.byref(c), ctypes.byref(i), ctypes.byref(ms)),
          "amr_hydro_box_tuning")
    return {"grid": g.value, "chunked": c.value, "interleave": i.value, "ms_per_step": ms.value}


def amr_hydro_step_adjoint(ctx, level, dt, U_n, lam_np1, lam_n):
    check(lib().amr_hydro_step_adjoint(ctx, level, dt, _p(U_n), _p(lam_np1), _p(lam_n)),
          "amr_hydro_step_adjoint")


def amr_hydro_uniform_tables(np_):
    """Host tables of a fully covered level: returns numpy int32 arrays
    (corner [n][3], sib [n][26], parent [n], child_group [n])."""
    import numpy as np
    n = int(np_[0]) * int(np_[1]) * int(np_[2])
    corner = np.empty((n, 3), np.int32)
    sib = np.empty((n, 26), np.int32)
    parent = np.empty(n, np.int32)
    child = np.empty(n, np.int32)
    dims = (ctypes.c_int * 3)(*[int(v) for v in np_])
    check(lib().amr_hydro_uniform_tables(dims, corner.ctypes.data, sib.ctypes.data, parent.ctypes.data,
                                         child.ctypes.data), "amr_hydro_uniform_tables")
    return corner, sib, parent, child


def amr_hydro_pack_uniform(dense, nx, ny, nz, patches, stream=None):
    check(lib().amr_hydro_pack_uniform(_p(dense), nx, ny, nz, _p(patches), _p(stream)),
          "amr_hydro_pack_uniform")


def amr_hydro_unpack_uniform(patches, nx, ny, nz, dense, stream=None):
    check(lib().amr_hydro_unpack_uniform(_p(patches), nx, ny, nz, _p(dense), _p(stream)),
          "amr_hydro_unpack_uniform")


def amr_hydro_advance_host(ctx, U_in, U_out, dt=-1.0):
    """One step of the uniform root grid from host state U_in to host state
    U_out ([5][nz][ny][nx] float64, page-locked for overlapped copies);
    returns the CFL dt of U_out."""
    dn = ctypes.c_double()
    check(lib().amr_hydro_advance_host(ctx, _p(U_in), _p(U_out), dt, ctypes.byref(dn)), "amr_hydro_advance_host")
    return dn.value


def amr_hydro_step_uniform_noalloc(U_old, U_new, nx, ny, nz, dh, dt, gamma, cfl, prec,
                                   dt_next_out=None, n_unphysical_out=None, stream=None):
    """One uniform periodic step with no device allocation (static scratch)."""
    check(lib().amr_hydro_step_uniform_noalloc(_p(U_old), _p(U_new), nx, ny, nz, dh, dt, gamma, cfl, prec,
                                               _p(dt_next_out), _p(n_unphysical_out), _p(stream)),
          "amr_hydro_step_uniform_noalloc")


def amr_hydro_bind_level(ctx, level, U_a, U_b, corner, sib, parent, child_group):
    check(lib().amr_hydro_bind_level(ctx, level, _p(U_a), _p(U_b), _p(corner), _p(sib), _p(parent),
                                     _p(child_group)), "amr_hydro_bind_level")


def amr_hydro_regrid(ctx, level):
    check(lib().amr_hydro_regrid(ctx, level), "amr_hydro_regrid")


def amr_hydro_advance_root(ctx, dt0=-1.0):
    """One root step of the W-cycle; returns the number of cell updates."""
    n = ctypes.c_int64()
    check(lib().amr_hydro_advance_root(ctx, dt0, ctypes.byref(n)), "amr_hydro_advance_root")
    return n.value


def amr_hydro_level_info(ctx, level):
    n, g = ctypes.c_int(), ctypes.c_int()
    check(lib().amr_hydro_level_info(ctx, level, ctypes.byref(n), ctypes.byref(g)), "amr_hydro_level_info")
    return n.value, g.value


def make_params(gamma=5.0 / 3.0, cfl=0.5, root_n=(64, 64, 64), box=None, lmax=0,
                prec=AMR_FP64, max_patches=None, theta=0.05, c_inc=0.1, c_dec=0.1, nbuf=None,
                limiter=AMR_LIM_VANLEER, riemann=AMR_RS_HLLC, minmod_coeff=1.5, scheme=AMR_SCHEME_MH,
                recon=AMR_RECON_PLM, fallback=0, dt_min=0.0, dual_energy=0, dual_xi=0.0,
                gravity_bc=AMR_GRAVITY_PERIODIC):
    p = amr_hydro_params()
    p.limiter, p.riemann, p.minmod_coeff, p.scheme, p.recon = limiter, riemann, minmod_coeff, scheme, recon
    p.fallback, p.dt_min, p.dual_energy, p.dual_xi = fallback, dt_min, dual_energy, dual_xi
    p.gravity_bc = gravity_bc
    p.gamma, p.cfl, p.c_inc, p.c_dec, p.theta = gamma, cfl, c_inc, c_dec, theta
    p.lmax = lmax
    nb = nbuf if nbuf is not None else [8] * 8
    for i in range(8):
        p.nbuf[i] = nb[i] if i < len(nb) else 8
    p.prec = prec
    for d in range(3):
        p.periodic[d] = 1
        p.root_n[d] = root_n[d]
        p.box[d] = (box[d] if box is not None else root_n[d] / root_n[0])
    if max_patches is None:
        max_patches = (root_n[0] // 8) * (root_n[1] // 8) * (root_n[2] // 8)
    p.max_patches = max_patches
    return p


def amr_hydro_phase_timing(ctx, on=True):
    check(lib().amr_hydro_phase_timing(ctx, 1 if on else 0), "amr_hydro_phase_timing")


def amr_hydro_phase_times(ctx):
    """{phase name: (ms, calls)} since the last call (synchronises the stream)."""
    ms = (ctypes.c_double * AMR_N_PHASES)()
    n = (ctypes.c_int64 * AMR_N_PHASES)()
    check(lib().amr_hydro_phase_times(ctx, ms, n), "amr_hydro_phase_times")
    return {PHASE_NAMES[k]: (ms[k], n[k]) for k in range(AMR_N_PHASES)}


def amr_hydro_set_box_entropy(ctx, box_id, S_a, S_b):
    check(lib().amr_hydro_set_box_entropy(ctx, box_id, _p(S_a), _p(S_b)), "amr_hydro_set_box_entropy")


def amr_hydro_set_shared_dt(ctx, on):
    check(lib().amr_hydro_set_shared_dt(ctx, 1 if on else 0), "amr_hydro_set_shared_dt")


def amr_hydro_set_gravity(ctx, G, omega=1.7, iters=60, acc_order=2):
    check(lib().amr_hydro_set_gravity(ctx, G, omega, iters, acc_order), "amr_hydro_set_gravity")


def amr_hydro_level_gravity(ctx, level, phi_out=None, acc_out=None):
    check(lib().amr_hydro_level_gravity(ctx, level, _p(phi_out), _p(acc_out)), "amr_hydro_level_gravity")
