"""The host planning of z-runs (work items of the step kernel: chains of
same-level patch groups stacked in z), on the CPU: every group in exactly one
run, runs no longer than asked, consecutive groups of a run stacked in z, on
synthetic neighbour links (chains, a singleton, a periodic cycle, a
self-link) and on uniform periodic levels."""
import ctypes

import numpy as np
import pytest

from paper_1712_07070_b300 import amr_hydro as A

_i32p = ctypes.POINTER(ctypes.c_int32)


def runs_of(nbr, n_groups, max_len):
    fn = A.lib().amrh_selftest_runs
    fn.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, _i32p, _i32p]
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    runs = np.full(n_groups, -1, np.int32)
    off = np.full(n_groups + 1, -1, np.int32)
    n = fn(n_groups, nbr.ctypes.data_as(_i32p), max_len, runs.ctypes.data_as(_i32p), off.ctypes.data_as(_i32p))
    return [runs[off[i]:off[i + 1]].tolist() for i in range(n)]


def linked(n_groups, ups):
    """A neighbour plan whose only entries are the z links g -> u (position 53
    of g holds u's first patch, position 5 of u holds g's patch (0,0,1))."""
    nbr = np.full((n_groups, 64), -1, np.int32)
    for g, u in ups.items():
        nbr[g, 53] = 8 * u
        nbr[u, 5] = 8 * g + 4
    return nbr


def test_synthetic_chains_cycle_and_self_link():
    ups = {0: 3, 3: 7, 1: 2, 5: 6, 6: 5, 8: 9, 10: 10}
    runs = runs_of(linked(11, ups), 11, 2)
    # chains from groups without a lower neighbour, in group order, then the cycle
    assert runs == [[0, 3], [7], [1, 2], [4], [8, 9], [10], [5, 6]]
    runs = runs_of(linked(11, ups), 11, 16)
    assert runs == [[0, 3, 7], [1, 2], [4], [8, 9], [10], [5, 6]]


def test_one_sided_link_is_not_followed():
    nbr = linked(3, {0: 1})
    nbr[1, 5] = -1  # 1 does not see 0 below it
    assert runs_of(nbr, 3, 4) == [[0], [1], [2]]


@pytest.mark.parametrize("np_,max_len", [((4, 6, 8), 3), ((8, 4, 2), 16), ((2, 2, 32), 5), ((4, 4, 4), 1)])
def test_uniform_level_runs_are_z_columns(np_, max_len):
    corner, sib, parent, child = A.amr_hydro_uniform_tables(np_)
    n_patches = len(corner)
    ng = n_patches // 8
    fn = A.lib().amrh_selftest_nbr_plan
    fn.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i32p, _i32p, _i32p]
    cells = (ctypes.c_int * 3)(*(8 * n for n in np_))
    nbr = np.zeros((ng, 64), np.int32)
    assert fn(0, n_patches, corner.ctypes.data_as(_i32p), sib.ctypes.data_as(_i32p), None,
              ctypes.cast(cells, _i32p), nbr.ctypes.data_as(_i32p)) == 0
    runs = runs_of(nbr, ng, max_len)
    flat = [g for r in runs for g in r]
    assert sorted(flat) == list(range(ng))
    ngx, ngy, ngz = np_[0] // 2, np_[1] // 2, np_[2] // 2
    for r in runs:
        assert 1 <= len(r) <= max_len
        for a, b in zip(r, r[1:]):
            assert b == (a + ngx * ngy) % ng  # the group directly above (periodic in z)
    if ngz > 1:  # each z column is one cycle, cut into runs of max_len
        assert len(runs) == ngx * ngy * -(-ngz // max_len)
    else:  # a single group per column is its own upper neighbour: no link
        assert len(runs) == ng


@pytest.mark.parametrize("chains,grid,e,expect", [
    ([16] * 256, 148, 0.05, 4),    # 256^3 FP64: 1024 runs in 7 rounds of 4.05
    ([32] * 1024, 296, 0.13, 16),  # 512^3 FP32 mode: 2048 runs in 7 rounds of 16.13
    ([16] * 256, 296, 0.13, 2),    # 256^3 FP32 mode: 2048 runs in 7 rounds of 2.13
    ([1] * 500, 148, 0.05, 1),     # no stacked groups: single-group runs
])
def test_run_length_choice(chains, grid, e, expect):
    """The round-robin cost estimate ceil(n_runs / grid) (len + e) picks the
    lengths that measured fastest on those levels."""
    fn = A.lib().amrh_selftest_run_len
    fn.argtypes = [ctypes.c_int, _i32p, ctypes.c_int, ctypes.c_double]
    L = np.array(chains, np.int32)
    assert fn(len(L), L.ctypes.data_as(_i32p), grid, e) == expect
