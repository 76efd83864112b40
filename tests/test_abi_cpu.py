"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol include/amr_hydro.h declares, validates parameters before any
device work, and builds correct uniform-level tables (section 2.1: every
patch stores its 26 sibling ids)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1712_07070_b300 import amr_hydro as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "amr_hydro.h")).read()
    return sorted(set(re.findall(r"\b(amr_hydro_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = A.lib()
    decl = declared_symbols()
    assert len(decl) >= 18
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(A.SYMBOLS) == decl


def test_every_symbol_has_declared_argument_types():
    # an undeclared signature would pass 64-bit pointers as C ints
    L = A.lib()
    for name in A.SYMBOLS:
        assert getattr(L, name).argtypes is not None, name


def test_strerror():
    assert A.strerror(A.AMR_OK) == "ok"
    assert "unphysical" in A.strerror(A.AMR_E_UNPHYSICAL)


@pytest.mark.parametrize("field,value", [("gamma", 1.0), ("cfl", 0.0), ("lmax", 9), ("max_patches", 12),
                                         ("prec", 7), ("limiter", 4), ("limiter", -1), ("riemann", 4),
                                         ("minmod_coeff", 0.5), ("minmod_coeff", 2.5), ("scheme", 3),
                                         ("scheme", -1), ("recon", 2), ("recon", -1), ("fallback", 2),
                                         ("dt_min", -1.0), ("dual_energy", 2), ("dual_xi", -1.0),
                                         ("gravity_bc", 2), ("gravity_bc", -1)])
def test_init_rejects_bad_params(field, value):
    p = A.make_params(root_n=(32, 32, 32))
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    assert A.lib().amr_hydro_init(ctypes.byref(p), None, ctypes.byref(ctx)) == A.AMR_E_INVAL
    assert not ctx.value


def test_init_rejects_vl_with_ppm():
    # the VL scheme reconstructs its half step with PLM only
    ctx = ctypes.c_void_p()
    p = A.make_params(root_n=(32, 32, 32), scheme=A.AMR_SCHEME_VL, recon=A.AMR_RECON_PPM)
    assert A.lib().amr_hydro_init(ctypes.byref(p), None, ctypes.byref(ctx)) == A.AMR_E_INVAL
    assert not ctx.value


def test_init_rejects_dual_energy_outside_its_scope():
    # built for MUSCL-Hancock + PLM without the cell remedies
    ctx = ctypes.c_void_p()
    for kw in (dict(scheme=A.AMR_SCHEME_CTU), dict(scheme=A.AMR_SCHEME_VL), dict(recon=A.AMR_RECON_PPM),
               dict(fallback=1)):
        p = A.make_params(root_n=(32, 32, 32), dual_energy=1, **kw)
        assert A.lib().amr_hydro_init(ctypes.byref(p), None, ctypes.byref(ctx)) == A.AMR_E_INVAL, kw
        assert not ctx.value


def test_init_rejects_non_multiple_of_16_and_non_cubic_cells():
    p = A.make_params(root_n=(40, 32, 32))
    ctx = ctypes.c_void_p()
    assert A.lib().amr_hydro_init(ctypes.byref(p), None, ctypes.byref(ctx)) == A.AMR_E_INVAL
    p = A.make_params(root_n=(32, 32, 32), box=(1.0, 2.0, 1.0))
    assert A.lib().amr_hydro_init(ctypes.byref(p), None, ctypes.byref(ctx)) == A.AMR_E_INVAL
    p = A.make_params(root_n=(32, 32, 32))
    p.periodic[1] = 0
    assert A.lib().amr_hydro_init(ctypes.byref(p), None, ctypes.byref(ctx)) == A.AMR_E_INVAL


@pytest.mark.parametrize("np_", [(2, 2, 2), (4, 2, 6), (8, 8, 8)])
def test_uniform_tables_match_brute_force(np_):
    corner, sib, parent, child = A.amr_hydro_uniform_tables(np_)
    n = np.prod(np_)
    assert (parent == -1).all() and (child == -1).all()
    # corners are a permutation of all patch positions; groups are 2x2x2 blocks
    pos = corner // 8
    assert len({tuple(p) for p in pos}) == n
    for g in range(n // 8):
        blk = pos[8 * g:8 * g + 8]
        base = blk[0]
        assert (base % 2 == 0).all()
        for l in range(8):
            assert tuple(blk[l] - base) == (l & 1, (l >> 1) & 1, (l >> 2) & 1)
    lookup = {tuple(p): s for s, p in enumerate(pos)}
    k = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx == dy == dz == 0:
                    continue
                for s in range(n):
                    q = (pos[s] + np.array([dx, dy, dz])) % np.array(np_)
                    assert sib[s, k] == lookup[tuple(q)]
                k += 1


def test_uniform_tables_reject_odd_counts():
    with pytest.raises(A.AmrHydroError):
        A.amr_hydro_uniform_tables((3, 2, 2))


def test_null_context_calls_are_rejected():
    # entry points that take a context check it before any CUDA work
    L = A.lib()
    assert L.amr_hydro_set_shared_dt(None, 1) == A.AMR_E_INVAL
    assert L.amr_hydro_regrid(None, 0) == A.AMR_E_INVAL
    assert L.amr_hydro_set_gravity(None, 1.0, 1.7, 10, 2) == A.AMR_E_INVAL
