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


# ---- coarse-fine time interpolation (section 3.2 ghosts; section 2.1 adaptive steps) ----

def _linear_fields(n, a):
    """Two different linear conserved fields at the cell centres of an n^3
    grid: a = 0 and a = 1 give the coarse level's old and new states."""
    x, y, z = ics.grid(n)
    rho = 2.0 + (0.3 + 0.5 * a) * x - (0.2 - 0.1 * a) * y + 0.1 * z
    return np.stack([rho, 0.05 * x + 0.2 * a, -0.02 * y - 0.1 * a * z, 0.01 * z + 0.03 + 0.04 * a * x,
                     10.0 + x + 2 * y - z + 3.0 * a * y])


def _one_group_hierarchy(U_old, U_new, t_old, t_new):
    H = OA.OracleHierarchy(np.ascontiguousarray(U_new), lmax=1, gamma=G53, cfl=0.5, theta=0.05, nbuf=[1],
                           regrid_at_start=False)
    H.lv[1].mask[1:3, 1:3, 1:3] = 1   # one group, fine cells 8..23 per dimension
    H.lv[1].U[:] = -7.0                # marker: fill_ghost must not touch patch cells
    c = H.lv[0]
    c.U_prev, c.U = np.ascontiguousarray(U_old), np.ascontiguousarray(U_new)
    c.t_prev, c.t = t_old, t_new
    return H


def _ghost_region():
    m = np.zeros((32, 32, 32), bool)
    m[5:27, 5:27, 5:27] = True        # within 3 cells of the group
    m[8:24, 8:24, 8:24] = False
    return m


def test_time_interpolation_hand_weight():
    # coarse level at t_old = 2.0 (field A) and t_new = 2.5 (field B); ghosts
    # of the fine level at t = 2.15 are the weight w = (2.15 - 2.0)/0.5 = 0.3
    # blend 0.7 A + 0.3 B; both fields are linear and the ghost parents'
    # stencils stay inside the domain, so the limited prolongation reproduces
    # them exactly and the ghost value is 0.7 A(x_f) + 0.3 B(x_f) at the fine
    # cell centre x_f.
    A_c, B_c = _linear_fields(16, 0.0), _linear_fields(16, 1.0)
    A_f, B_f = _linear_fields(32, 0.0), _linear_fields(32, 1.0)
    H = _one_group_hierarchy(A_c, B_c, 2.0, 2.5)
    H.fill_ghost(1, 2.15)
    g = _ghost_region()
    got = H.lv[1].U[:, g]
    want = 0.7 * A_f[:, g] + 0.3 * B_f[:, g]
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # old and new swapped (weight 1 - w) is far from it
    wrong = 0.3 * A_f[:, g] + 0.7 * B_f[:, g]
    assert np.abs(got - wrong).max() > 0.05
    # the patch cells are not ghosts
    assert (H.lv[1].U[:, 8:24, 8:24, 8:24] == -7.0).all()


def test_time_interpolation_exact_endpoints():
    # at t = t_old the ghosts are the prolongation of exactly the old field,
    # at t = t_new of exactly the new one (bitwise: no blend is formed)
    A_c = np.ascontiguousarray(ics.turbulence(16, seed=7))
    B_c = np.ascontiguousarray(ics.turbulence(16, seed=8))
    g = _ghost_region()
    full = np.ones((4, 4, 4), np.uint8)
    for t, src in ((2.0, A_c), (2.5, B_c)):
        H = _one_group_hierarchy(A_c, B_c, 2.0, 2.5)
        H.fill_ghost(1, t)
        assert np.array_equal(H.lv[1].U[:, g], prolong(src, full)[:, g])


# ---- cell refinement criterion (section 2.1: first-derivative criterion, normalised) ----

def _flags_of_density(rho, theta):
    n = rho.shape[0]
    U0 = np.stack([rho, 0 * rho, 0 * rho, 0 * rho, 1.0 + 0 * rho])
    H = OA.OracleHierarchy(np.ascontiguousarray(U0), lmax=1, gamma=G53, cfl=0.5, theta=theta, nbuf=[0],
                           regrid_at_start=False)
    return H.cell_flags(0)


def test_refinement_criterion_hand_values_1d():
    # rho along one axis of a periodic 8^3 level, theta = 1/2: the flag is
    # g^2 > theta^2 rho^2 with g = (rho_{i+1} - rho_{i-1})/2 (the other two
    # central differences vanish).  Hand evaluation, cell by cell:
    #   i : rho  g      g^2   theta^2 rho^2   flag
    #   0 : 1    0      0     0.25            0
    #   1 : 1    0.5    0.25  0.25            0   (equality: strict >)
    #   2 : 2    1      1     1               0   (equality)
    #   3 : 3   -0.5    0.25  2.25            0
    #   4 : 1   -1      1     0.25            1   (normalised by its own rho)
    #   5 : 1    1.5    2.25  0.25            1
    #   6 : 4    0      0     4               0
    #   7 : 1   -1.5    2.25  0.25            1   (wraps to cell 0)
    F = np.array([1.0, 1.0, 2.0, 3.0, 1.0, 1.0, 4.0, 1.0])
    want = np.array([0, 0, 0, 0, 1, 1, 0, 1], np.uint8)
    ones = np.ones((8, 8, 8))
    for axis in (2, 1, 0):  # x, y, z
        shape = [1, 1, 1]
        shape[axis] = 8
        rho = ones * F.reshape(shape)
        f = _flags_of_density(rho, 0.5)
        got = np.moveaxis(f, axis, 0)
        assert (got == want.reshape(8, 1, 1)).all(), (axis, got[:, 0, 0])


def test_refinement_criterion_sums_squares_over_dimensions():
    # rho = F((x + y) mod 8): on the cells with x + y = 2 (mod 8), rho = 2 and
    # both central differences are (3 - 1)/2 = 1, so g^2 = 2.  theta = 0.75
    # gives theta^2 rho^2 = 2.25 > 2 (not flagged; the squared L1 norm 4 would
    # flag it) and theta = 0.6 gives 1.44 < 2 (flagged; one dimension alone, 1,
    # would not).
    F = np.array([2.0, 1.0, 2.0, 3.0, 2.0, 2.0, 2.0, 2.0])
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    rho = F[(x + y) % 8]
    sel = (x + y) % 8 == 2
    assert not _flags_of_density(rho, 0.75)[sel].any()
    assert _flags_of_density(rho, 0.6)[sel].all()


# ---- adaptive time-step W-cycle (section 2.1 pseudo-code: C_inc and C_dec rules) ----

def _scripted_hierarchy(lmax, dts, shared_dt=False):
    """A hierarchy whose per-level CFL step comes from the scripted lists dts[l]
    (the last entry repeats) and whose level updates, fix-ups and regrids are
    only recorded: what is left is the W-cycle's control flow."""
    H = OA.OracleHierarchy(ics.uniform_state(16), lmax=lmax, gamma=G53, cfl=0.5, theta=0.05,
                           nbuf=[1] * lmax, regrid_at_start=False, shared_dt=shared_dt)
    for l in range(1, lmax + 1):
        H.lv[l].mask[0:2, 0:2, 0:2] = 1
    log, calls = [], [0] * (lmax + 1)

    def min_dt(l):
        k = min(calls[l], len(dts[l]) - 1)
        calls[l] += 1
        return dts[l][k]

    H.min_dt = min_dt
    H.advance_level = lambda l, dt: log.append(("step", l, dt))
    H.flux_fixup = lambda l: log.append(("fix", l))
    H.regrid = lambda l: log.append(("regrid", l))
    return H, log


def test_wcycle_dt_rule_two_levels_hand_sequence():
    # CFL steps: root 1, 17/16, 5/4, 1/2 in successive root steps; level 1
    # always 31/64.  C_inc = C_dec = 0.1.  Hand derivation:
    # root step 1: dt0 = 1 (no level-1 history).  Level 1 from t=0 to 1:
    #   31/64 (1.1*31/64 = 0.5328 < 1), then 1.1*31/64 > 1 - 31/64 = 33/64,
    #   so it lands: 33/64 (C_inc, a 6.5% longer step).
    # root step 2: CFL 17/16 > 2*(33/64) = 33/32 and 0.9*17/16 = 0.956 < 33/32:
    #   C_dec shrinks dt0 to 33/32.  Level 1 from 1 to 65/32: 31/64, 31/64
    #   (1.1*31/64 < 35/64), then the remaining 1/16 (C_inc).
    # root step 3: CFL 5/4 > 2/16 but 0.9*5/4 >= 1/8: unchanged, 5/4.  Level 1
    #   from 65/32 to 105/32: 31/64, 31/64, then the remaining 9/32.
    # root step 4: CFL 1/2 <= 2*(9/32) = 9/16: unchanged (never raised).  Level
    #   1: 1.1*31/64 > 1/2, so one step of exactly 1/2 (C_inc).
    H, log = _scripted_hierarchy(1, [[1.0, 17 / 16, 5 / 4, 1 / 2], [31 / 64]])
    for _ in range(4):
        H.advance(0)
    steps = [(e[1], e[2]) for e in log if e[0] == "step"]
    assert steps == [(0, 1.0), (1, 31 / 64), (1, 33 / 64),
                     (0, 33 / 32), (1, 31 / 64), (1, 31 / 64), (1, 1 / 16),
                     (0, 5 / 4), (1, 31 / 64), (1, 31 / 64), (1, 9 / 32),
                     (0, 1 / 2), (1, 1 / 2)]
    assert H.lv[0].t == H.lv[1].t == 1 + 33 / 32 + 5 / 4 + 1 / 2
    # after each level-1 sub-cycle: fix-up then regrid of level 0, once per root step
    assert [e for e in log if e[0] != "step"] == [("fix", 0), ("regrid", 0)] * 4


def test_wcycle_c_inc_takes_priority_over_c_dec():
    # Three levels.  Root CFL 17/16; level 1: 1/2 then 17/32; level 2: 1/4.
    # Level 1, first step: 1/2 (1.1/2 < 17/16; no level-2 history).  Level 2
    #   from 0 to 1/2: 1/4, then 1.1/4 > 1/4 lands exactly 1/4.
    # Level 1, second step: CFL 17/32 with 17/16 - 1/2 = 9/16 left: the C_inc
    #   test 1.1*17/32 = 0.584 > 9/16 holds, and so does the C_dec test
    #   (17/32 > 2*(1/4) and 0.9*17/32 < 1/2); the pseudo-code's "else if"
    #   makes C_inc win: the step is 9/16, not 1/2.  Level 2 from 1/2 to
    #   17/16: 1/4, 1/4, then the remaining 1/16.
    H, log = _scripted_hierarchy(2, [[17 / 16], [1 / 2, 17 / 32], [1 / 4]])
    H.advance(0)
    assert log == [("step", 0, 17 / 16),
                   ("step", 1, 1 / 2), ("step", 2, 1 / 4), ("step", 2, 1 / 4), ("fix", 1), ("regrid", 1),
                   ("step", 1, 9 / 16), ("step", 2, 1 / 4), ("step", 2, 1 / 4), ("step", 2, 1 / 16),
                   ("fix", 1), ("regrid", 1),
                   ("fix", 0), ("regrid", 0)]
    assert H.lv[0].t == H.lv[1].t == H.lv[2].t == 17 / 16


# ---- shared time-step integration (section 2.6: the constraints of all levels, the minimum) ----

def test_shared_dt_takes_the_minimum_over_levels_one_step_each():
    # CFL steps: root 1 then 1/4; level 1 1/2; level 2 3/8 then 5/8.
    # Root step 1: min(1, 1/2, 3/8) = 3/8 on every level, one step each (the
    #   level's own step 1/2 or 5/8 is never taken).  Root step 2: the
    #   constraints are evaluated again on all levels: min(1/4, 1/2, 5/8) = 1/4.
    # No C_dec rule: in the adaptive cycle root step 2's 1/4 < 2*(3/8) keeps
    # its value anyway, and step 1 checks the rule's absence below.
    H, log = _scripted_hierarchy(2, [[1.0, 1 / 4], [1 / 2], [3 / 8, 5 / 8]], shared_dt=True)
    for _ in range(2):
        H.advance(0)
    assert log == [("step", 0, 3 / 8), ("step", 1, 3 / 8), ("step", 2, 3 / 8), ("fix", 1), ("regrid", 1),
                   ("fix", 0), ("regrid", 0),
                   ("step", 0, 1 / 4), ("step", 1, 1 / 4), ("step", 2, 1 / 4), ("fix", 1), ("regrid", 1),
                   ("fix", 0), ("regrid", 0)]
    assert H.lv[0].t == H.lv[1].t == H.lv[2].t == 3 / 8 + 1 / 4


def test_shared_dt_applies_no_c_dec_shrink():
    # root CFL 17/16 with level 1's previous step 33/64: the adaptive cycle
    # shrinks the root step to 2*(33/64) = 33/32 (C_dec; see the hand
    # sequence above), the shared one keeps the minimum over levels, 17/16
    # when level 1's own constraint (9/8) is larger
    for shared, want in ((False, 33 / 32), (True, 17 / 16)):
        H, log = _scripted_hierarchy(1, [[17 / 16], [9 / 8]], shared_dt=shared)
        H.lv[1].dt_prev = 33 / 64
        H.advance(0)
        steps = [(e[1], e[2]) for e in log if e[0] == "step"]
        assert steps[0] == (0, want), (shared, steps)
        if shared:
            assert steps == [(0, 17 / 16), (1, 17 / 16)]


def test_shared_dt_hierarchy_keeps_levels_in_step_and_conserves():
    U0 = ics.blobs(32, seed=5, contrast=10.0, mach=1.0)
    H = OA.OracleHierarchy(U0, lmax=2, gamma=G53, cfl=0.5, theta=0.3, nbuf=[1, 1], shared_dt=True)
    assert not H.lv[2].empty

    def mass():
        return sum(H.lv[l].U[0][H.leaf(l)].sum() * H.dh(l) ** 3 for l in range(3) if not H.lv[l].empty)

    m0 = mass()
    for _ in range(2):
        own = [H.min_dt(l) for l in range(3) if not H.lv[l].empty]
        n0 = len(H.log)
        H.advance(0)
        steps = H.log[n0:]
        assert [l for l, _ in steps] == [0, 1, 2]
        assert steps[0][1] == min(own) and min(own) < max(own)
        assert H.lv[0].t == H.lv[1].t == H.lv[2].t
    assert abs(mass() - m0) <= 1e-14 * m0
