"""Pins of the AMR oracle (section 2.1 hierarchy and regrid rules, section
2.2 restriction and flux fix-up, section 3.2 coarse-fine interpolation)
against facts fixed independently of it: exactness on linear fields,
conservation of the prolongation, equivalence of a fully refined level with
a uniform run at its resolution, conservation across fix-up and regrid, and
hand-derived hierarchies for hand-made flag sets."""
import numpy as np
import pytest

import oracle
from oracle import amr as OA
from paper_1712_07070_b300 import ics

G53 = 5.0 / 3.0


def linear_state(n):
    x, y, z = ics.grid(n)
    rho = 2.0 + 0.3 * x - 0.2 * y + 0.1 * z
    return np.stack([rho, 0.05 * x, -0.02 * y, 0.01 * z + 0.03, 10.0 + x + 2 * y - z])


def prolong(Uc, newmask):
    Nc = Uc.shape[-1]
    Nf = 2 * Nc
    Uf = np.zeros((5, Nf, Nf, Nf))
    OA.amr_lib().or_amr_prolong_patches(oracle._ptr(Uf), OA._u8(newmask), OA._dims([Nf] * 3), oracle._ptr(Uc))
    return Uf


def test_prolongation_exact_on_linear_fields():
    Uc = linear_state(16)
    mask = np.zeros((4, 4, 4), np.uint8)
    mask[1:3, 1:3, 1:3] = 1  # interior patches, away from the periodic wrap
    Uf = prolong(np.ascontiguousarray(Uc), mask)
    exact = linear_state(32)
    cm = OA.cell_mask(mask)
    assert np.abs(Uf[:, cm] - exact[:, cm]).max() < 1e-13


def test_prolongation_conservative_and_positive():
    rng = np.random.default_rng(1)
    Uc = ics.blobs(16, seed=3)  # strong blobs: triggers the positivity fallback somewhere
    mask = np.ones((4, 4, 4), np.uint8)
    Uf = prolong(np.ascontiguousarray(Uc), mask)
    mean = Uf.reshape(5, 16, 2, 16, 2, 16, 2).mean(axis=(2, 4, 6))
    assert np.abs(mean - Uc).max() <= 1e-13 * np.abs(Uc).max()
    rho = Uf[0]
    P = (G53 - 1) * (Uf[4] - 0.5 * (Uf[1] ** 2 + Uf[2] ** 2 + Uf[3] ** 2) / rho)
    assert (rho > 0).all() and (P > 0).all()
    # and without the fallback the same interpolation would not be positive
    assert not np.isclose(Uf, np.repeat(np.repeat(np.repeat(Uc, 2, 1), 2, 2), 2, 3)).all()


def test_restriction_of_prolongation_is_identity():
    Uc = np.ascontiguousarray(ics.turbulence(16, seed=2))
    mask = np.ones((4, 4, 4), np.uint8)
    Uf = prolong(Uc, mask)
    Ur = np.zeros_like(Uc)
    cov = np.ones((16, 16, 16), np.uint8)
    OA.amr_lib().or_amr_restrict(oracle._ptr(Ur), oracle._ptr(Uf), OA._u8(cov), OA._dims([16] * 3))
    assert np.abs(Ur - Uc).max() <= 1e-14 * np.abs(Uc).max()


def test_fully_refined_level_equals_uniform_run():
    # theta=0 flags every cell with a nonzero density gradient: level 1 covers
    # the whole domain, has all its siblings, and so must evolve exactly like
    # a uniform run at its resolution from the same (prolonged) data with the
    # same time steps
    U0 = ics.sod_noise(16, seed=4)
    H = OA.OracleHierarchy(U0, lmax=1, gamma=G53, cfl=0.5, theta=0.0, nbuf=[8])
    assert H.lv[1].mask.all()
    Ustart = H.lv[1].U.copy()
    H.advance(0)
    H.advance(0)
    dts = [dt for (l, dt) in H.log if l == 1]
    assert len(dts) >= 4
    U = Ustart
    for dt in dts:
        U, nbad = oracle.step_periodic(U, 1.0 / 32, dt, G53)
    assert np.array_equal(U, H.lv[1].U)
    # and the root is the restriction of level 1
    mean = U.reshape(5, 16, 2, 16, 2, 16, 2).mean(axis=(2, 4, 6))
    assert np.abs(mean - H.lv[0].U).max() <= 1e-14 * np.abs(U).max()


def test_conservation_across_fixup_and_regrid():
    U0 = ics.blobs(32, seed=5, contrast=10.0, mach=1.0)
    H = OA.OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.05, nbuf=[8, 4])
    assert not H.lv[2].empty
    s0 = H.conserved_total()
    H.advance(0)
    s1 = H.conserved_total()
    scale = np.abs(U0).reshape(5, -1).sum(1) / 32 ** 3
    assert (np.abs(s1 - s0) <= 1e-13 * scale).all(), (s1 - s0) / scale


def test_fixup_matters():
    # without the fix-up the coarse-fine interface leaks mass: the pin above
    # would fail if the flux registers were dropped
    U0 = ics.blobs(32, seed=5, contrast=10.0, mach=1.0)
    H = OA.OracleHierarchy(U0, lmax=1, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1])
    assert 0 < H.lv[1].mask.sum() < H.lv[1].mask.size  # a real coarse-fine interface
    s0 = H.conserved_total()
    H.flux_fixup = lambda l: OA.amr_lib().or_amr_restrict(
        oracle._ptr(H.lv[l].U), oracle._ptr(H.lv[l + 1].U),
        OA._u8(OA.covered(H.lv[l + 1].mask, H.lv[l + 1].N)), OA._dims(H.lv[l].N))
    H.advance(0)
    s1 = H.conserved_total()
    assert abs(s1[1] - s0[1]) > 1e-9 * np.abs(U0[1]).sum() / 32 ** 3


# ---- bookkeeping on hand-made flag sets ---------------------------------------------

def quiet_hierarchy(n=32, lmax=2, nbuf=(4, 2)):
    U0 = ics.uniform_state(n)
    return OA.OracleHierarchy(U0, lmax=lmax, gamma=G53, cfl=0.5, theta=0.05, nbuf=list(nbuf),
                              regrid_at_start=False)


def patch_set(mask):
    return {tuple(int(v) for v in p[::-1]) for p in np.argwhere(mask.astype(bool))}  # (px,py,pz)


def test_single_flagged_cell_at_patch_corner():
    H = quiet_hierarchy()
    cf = np.zeros((32, 32, 32), np.uint8)
    cf[7, 7, 7] = 1  # cell (x,y,z)=(7,7,7): corner of patch (0,0,0); nbuf 4 reaches patches 0..1
    H.regrid(0, cell_flags=cf)
    expect_coarse = {(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)}
    expect = {(2 * a + i, 2 * b + j, 2 * c + k) for (a, b, c) in expect_coarse
              for i in (0, 1) for j in (0, 1) for k in (0, 1)}
    assert patch_set(H.lv[1].mask) == expect


def test_flag_buffer_wraps_periodically():
    H = quiet_hierarchy()
    cf = np.zeros((32, 32, 32), np.uint8)
    cf[0, 0, 0] = 1  # the buffer [-4, 4] wraps to the last patch in every dimension
    H.regrid(0, cell_flags=cf)
    coarse = {(a, b, c) for a in (3, 0) for b in (3, 0) for c in (3, 0)}
    assert patch_set(H.lv[1].mask) == {(2 * a + i, 2 * b + j, 2 * c + k) for (a, b, c) in coarse
                                       for i in (0, 1) for j in (0, 1) for k in (0, 1)}


def test_nesting_rejects_refinement_at_level_edge_and_keeps_parents():
    H = quiet_hierarchy(nbuf=(0, 0))
    cf = np.zeros((32, 32, 32), np.uint8)
    cf[12:20, 12:20, 12:20] = 1  # cells of root patches 1..2 in each dimension
    H.regrid(0, cell_flags=cf)
    lvl1 = patch_set(H.lv[1].mask)
    assert lvl1 == {(i, j, k) for i in range(2, 6) for j in range(2, 6) for k in range(2, 6)}
    # level-1 flags on an edge patch (2,2,2) and on an interior patch (3,3,3):
    # only the interior one has all 26 siblings on level 1
    cf1 = np.zeros((64, 64, 64), np.uint8)
    cf1[16, 16, 16] = 1   # patch (2,2,2)
    cf1[24, 24, 24] = 1   # patch (3,3,3)
    H.regrid(1, cell_flags=cf1)
    assert patch_set(H.lv[2].mask) == {(6 + i, 6 + j, 6 + k) for i in (0, 1) for j in (0, 1) for k in (0, 1)}
    # a root regrid with no flags must keep the level-1 parents of level 2
    # (patch (3,3,3) has children) and the level-1 patches around it
    H.regrid(0, cell_flags=np.zeros((32, 32, 32), np.uint8))
    lvl1b = patch_set(H.lv[1].mask)
    assert (3, 3, 3) in lvl1b
    need = {((3 + a) // 2, (3 + b) // 2, (3 + c) // 2) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}
    assert lvl1b == {(2 * a + i, 2 * b + j, 2 * c + k) for (a, b, c) in need
                     for i in (0, 1) for j in (0, 1) for k in (0, 1)}
