// host_plan.cpp -- host-side planning of a level's patch-group gathers
// (GAMER-2 section 2.1: octree of 8^3 patches storing parent, child and 26
// sibling ids; section 3.1: patch groups of 8 siblings are the unit of work).
#include <cstdint>
#include <vector>

#include "ctx.h"

namespace amrh {

static inline int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

static inline int sib_index(int dx, int dy, int dz) {
    const int k = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
    return k - (k > 13);
}

amr_status build_uniform_tables(const int np[3], int32_t *corner, int32_t *sib, int32_t *parent,
                                int32_t *child) {
    for (int d = 0; d < 3; d++)
        if (np[d] <= 0 || np[d] % 2) return AMR_E_INVAL;
    const int ng[3] = {np[0] / 2, np[1] / 2, np[2] / 2};
    auto slot_of = [&](int px, int py, int pz) -> int32_t {
        px = wrapi(px, np[0]);
        py = wrapi(py, np[1]);
        pz = wrapi(pz, np[2]);
        const int64_t g = (px >> 1) + (int64_t)ng[0] * ((py >> 1) + (int64_t)ng[1] * (pz >> 1));
        return (int32_t)(8 * g + (px & 1) + 2 * (py & 1) + 4 * (pz & 1));
    };
    for (int pz = 0; pz < np[2]; pz++)
        for (int py = 0; py < np[1]; py++)
            for (int px = 0; px < np[0]; px++) {
                const int32_t s = slot_of(px, py, pz);
                corner[3 * s + 0] = 8 * px;
                corner[3 * s + 1] = 8 * py;
                corner[3 * s + 2] = 8 * pz;
                if (parent) parent[s] = -1;
                if (child) child[s] = -1;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            if (!dx && !dy && !dz) continue;
                            sib[26 * (int64_t)s + sib_index(dx, dy, dz)] = slot_of(px + dx, py + dy, pz + dz);
                        }
            }
    return AMR_OK;
}

// For every group, the source of each of the 4x4x4 patch positions around
// it (position q in {-1,0,1,2}^3, index (qx+1) + 4(qy+1) + 16(qz+1)):
//   >= 0   a same-level slot,
//   <= -2  coarse-fine ghost patch number (-2 - value), to be interpolated,
//   -1     a corner position, which no stencil of the step reads.
// Fails with AMR_E_NESTING when a face or edge neighbour is missing on the
// root level (nothing to interpolate from).  ghost_depth (even: 2 for PLM, 4
// for PPM's three ghost cells) is how deep the interpolated box of a ghost
// patch reaches along an outer direction; with corners, corner positions get
// ghost patches too (the per-cell remedies read a cell's 3x3x3 block).
amr_status build_nbr_plan(int level, int n_patches, const int32_t *corner, const int32_t *sib,
                          const int32_t *parent, const int level_cells[3],
                          std::vector<int32_t> &nbr, std::vector<GhostInfo> &ghosts, int ghost_depth,
                          bool corners) {
    const int n_groups = n_patches / 8;
    nbr.assign((size_t)n_groups * 64, -1);
    ghosts.clear();
    // per position (qx+1) + 4(qy+1) + 16(qz+1): the group's own patch it is
    // reached from, the sibling index of the step to it, its offset in cells,
    // whether it is a corner (never read) and the box of its cells the
    // group's stencils reach (ghost_depth deep along an outer direction, all 8
    // along an inner one)
    struct PosInfo {
        int own, sk, off[3], corner, box;
    };
    PosInfo pi[64];
    for (int pos = 0; pos < 64; pos++) {
        const int q3[3] = {(pos & 3) - 1, ((pos >> 2) & 3) - 1, (pos >> 4) - 1};
        int p3[3], d3[3], box = 0;
        for (int d = 0; d < 3; d++) {
            p3[d] = q3[d] < 0 ? 0 : (q3[d] > 1 ? 1 : q3[d]);
            d3[d] = q3[d] - p3[d];
            box |= (q3[d] < 0 ? 8 - ghost_depth : 0) << (4 * d) | (q3[d] > 1 ? ghost_depth : 8) << (12 + 4 * d);
        }
        PosInfo &e = pi[pos];
        e.own = p3[0] + 2 * p3[1] + 4 * p3[2];
        e.sk = (d3[0] || d3[1] || d3[2]) ? sib_index(d3[0], d3[1], d3[2]) : -1;
        for (int d = 0; d < 3; d++) e.off[d] = 8 * d3[d];
        e.corner = (d3[0] != 0) + (d3[1] != 0) + (d3[2] != 0) == 3;
        e.box = box;
    }
    // ghost patch ids by patch position (dense: the level's patch grid)
    const int P[3] = {level_cells[0] / 8, level_cells[1] / 8, level_cells[2] / 8};
    std::vector<int32_t> ghost_id;
    if (level > 0) ghost_id.assign((size_t)P[0] * P[1] * P[2], -1);
    auto wrapc = [](int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); };  // |step| <= one patch
    for (int g = 0; g < n_groups; g++) {
        int32_t *out = &nbr[(size_t)g * 64];
        for (int pos = 0; pos < 64; pos++) {
            const PosInfo &e = pi[pos];
            const int own = 8 * g + e.own;
            if (e.sk < 0) {
                out[pos] = own;
                continue;
            }
            const int32_t s = sib[26 * (int64_t)own + e.sk];
            if (s >= n_patches || s < -1) return AMR_E_INVAL;
            if (s >= 0) {
                out[pos] = s;
                continue;
            }
            if (e.corner && !corners) continue;  // read only by the cell remedies
            if (level == 0 || !parent) return AMR_E_NESTING;
            const int cx = wrapc(corner[3 * own + 0] + e.off[0], level_cells[0]);
            const int cy = wrapc(corner[3 * own + 1] + e.off[1], level_cells[1]);
            const int cz = wrapc(corner[3 * own + 2] + e.off[2], level_cells[2]);
            int32_t &slot_id = ghost_id[((size_t)(cz / 8) * P[1] + cy / 8) * P[0] + cx / 8];
            int id;
            if (slot_id < 0) {
                id = (int)ghosts.size();
                slot_id = id;
                GhostInfo gi;
                gi.cparent = parent[8 * g];
                gi.qx = (pos & 3) - 1;
                gi.qy = ((pos >> 2) & 3) - 1;
                gi.qz = (pos >> 4) - 1;
                gi.box = e.box;
                if (gi.cparent < 0) return AMR_E_NESTING;
                ghosts.push_back(gi);
            } else {
                id = slot_id;
                GhostInfo &gi = ghosts[id];  // union with what other groups read
                int b = gi.box;
                for (int d = 0; d < 3; d++) {
                    const int l0 = (b >> (4 * d)) & 15, h0 = (b >> (12 + 4 * d)) & 15;
                    const int ln = (e.box >> (4 * d)) & 15, hn = (e.box >> (12 + 4 * d)) & 15;
                    const int l1 = ln < l0 ? ln : l0, h1 = hn > h0 ? hn : h0;
                    b = (b & ~(15 << (4 * d)) & ~(15 << (12 + 4 * d))) | l1 << (4 * d) | h1 << (12 + 4 * d);
                }
                gi.box = b;
            }
            out[pos] = -2 - id;
        }
    }
    return AMR_OK;
}

// z-chains: group u is g's upper neighbour when position q = (0,0,2) of g
// (index 53) holds u's first patch and position q = (0,0,-1) of u (index 5)
// holds g's patch (0,0,1), i.e. both are same-level groups stacked in z.
// Chains follow the upper neighbours from groups with no lower neighbour (in
// group order), then the remaining cycles (periodic columns) from their
// lowest group.
void z_chains(int n_groups, const int32_t *nbr, std::vector<int32_t> &chains, std::vector<int32_t> &chain_off) {
    std::vector<int32_t> up(n_groups, -1), down(n_groups, -1);
    for (int g = 0; g < n_groups; g++) {
        const int32_t s = nbr[(size_t)g * 64 + 53];
        if (s < 0 || s % 8) continue;
        const int u = s / 8;
        if (u == g || u >= n_groups || nbr[(size_t)u * 64 + 5] != 8 * g + 4) continue;
        up[g] = u;
        down[u] = g;
    }
    chains.clear();
    chain_off.assign(1, 0);
    std::vector<char> seen(n_groups, 0);
    auto chain = [&](int g) {
        while (g >= 0 && !seen[g]) {
            seen[g] = 1;
            chains.push_back(g);
            g = up[g];
        }
        chain_off.push_back((int32_t)chains.size());
    };
    for (int g = 0; g < n_groups; g++)
        if (!seen[g] && down[g] < 0) chain(g);
    for (int g = 0; g < n_groups; g++)
        if (!seen[g]) chain(g);
}

// Each chain cut into runs of at most max_len groups, in chain order.
void cut_runs(const std::vector<int32_t> &chains, const std::vector<int32_t> &chain_off, int max_len,
              std::vector<int32_t> &runs, std::vector<int32_t> &run_off) {
    runs = chains;
    run_off.assign(1, 0);
    for (size_t c = 0; c + 1 < chain_off.size(); c++)
        for (int a = chain_off[c]; a < chain_off[c + 1]; a += max_len)
            run_off.push_back(a + max_len < chain_off[c + 1] ? a + max_len : chain_off[c + 1]);
}

void build_runs(int n_groups, const int32_t *nbr, int max_len, std::vector<int32_t> &runs,
                std::vector<int32_t> &run_off) {
    std::vector<int32_t> chains, off;
    z_chains(n_groups, nbr, chains, off);
    cut_runs(chains, off, max_len, runs, run_off);
}

// Run length for `grid` resident CTAs: the CTAs take runs round-robin, so a
// launch lasts about ceil(n_runs / grid) rounds of (len + e) group-steps,
// where e is the cost of a run beyond its groups (the two extra Hancock
// planes and four plane loads of its ends, its prologue; measured about 0.05
// group-steps in FP64 and 0.13 in the FP32 mode).  The length in 1..32 that
// minimises that estimate.
int choose_run_len(const std::vector<int32_t> &chain_off, int grid, double e) {
    int best_len = 1;
    double best = 1e300;
    for (int len = 1; len <= 32; len++) {
        long long n_runs = 0;
        int longest = 0;
        for (size_t c = 0; c + 1 < chain_off.size(); c++) {
            const int L = chain_off[c + 1] - chain_off[c];
            n_runs += (L + len - 1) / len;
            longest = L > longest ? L : longest;
        }
        const long long rounds = (n_runs + grid - 1) / grid;
        const double cost = (double)rounds * ((len < longest ? len : longest) + e);
        if (cost < best - 1e-9) {
            best = cost;
            best_len = len;
        }
    }
    return best_len;
}

}  // namespace amrh

extern "C" amr_status amr_hydro_uniform_tables(const int np[3], int32_t *corner, int32_t *sib,
                                               int32_t *parent, int32_t *child_group) {
    if (!np || !corner || !sib) return AMR_E_INVAL;
    return amrh::build_uniform_tables(np, corner, sib, parent, child_group);
}

// Test hook (not part of the C ABI): the z-runs build_runs makes for a
// neighbour plan; runs_out must hold n_groups entries and run_off_out
// n_groups + 1.  Returns the number of runs.
extern "C" int amrh_selftest_runs(int n_groups, const int32_t *nbr, int max_len, int32_t *runs_out,
                                  int32_t *run_off_out) {
    std::vector<int32_t> runs, off;
    amrh::build_runs(n_groups, nbr, max_len, runs, off);
    for (size_t i = 0; i < runs.size(); i++) runs_out[i] = runs[i];
    for (size_t i = 0; i < off.size(); i++) run_off_out[i] = off[i];
    return (int)off.size() - 1;
}

// Test hook: the neighbour plan of a level from host tables (corner, sib,
// parent as in amr_hydro_set_level); nbr_out: n_patches / 8 x 64 entries.
extern "C" int amrh_selftest_nbr_plan(int level, int n_patches, const int32_t *corner, const int32_t *sib,
                                      const int32_t *parent, const int level_cells[3], int32_t *nbr_out) {
    std::vector<int32_t> nbr;
    std::vector<amrh::GhostInfo> ghosts;
    const amr_status st = amrh::build_nbr_plan(level, n_patches, corner, sib, parent, level_cells, nbr, ghosts);
    if (st) return -1;
    for (size_t i = 0; i < nbr.size(); i++) nbr_out[i] = nbr[i];
    return (int)ghosts.size();
}

// Test hook: the run length choose_run_len picks for n_chains chains of the
// given lengths on `grid` resident CTAs with per-run overhead e.
extern "C" int amrh_selftest_run_len(int n_chains, const int32_t *lengths, int grid, double e) {
    std::vector<int32_t> off(1, 0);
    for (int c = 0; c < n_chains; c++) off.push_back(off.back() + lengths[c]);
    return amrh::choose_run_len(off, grid, e);
}
