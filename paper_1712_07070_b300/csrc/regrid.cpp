// regrid.cpp -- host-side AMR bookkeeping (GAMER-2 section 2.1):
//   * per-level gather plans and coarse-fine register maps;
//   * regridding one level at a time from device refinement flags: flag
//     buffers (on the device), proper nesting, no explicit derefinement
//     (children are removed when their parent is not flagged and no
//     grandchildren need them), new children interpolated from the parent;
//   * the adaptive time-step W-cycle with the C_inc / C_dec rule of the
//     section's pseudo-code, followed by fix-up (section 2.2) and regrid.
// Integer work only; all cell data moves on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <vector>

#include "amr_hydro.h"
#include "ctx.h"

namespace amrh {

constexpr int PSLOT_H = 5 * 512;

static inline int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}
static inline int sib_k(int dx, int dy, int dz) {
    const int k = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
    return k - (k > 13);
}
// face f (0..5: -x,+x,-y,+y,-z,+z) -> sibling index of the neighbour across it
static inline int face_sib(int f) {
    int d[3] = {0, 0, 0};
    d[f >> 1] = (f & 1) ? 1 : -1;
    return sib_k(d[0], d[1], d[2]);
}

template <typename T>
static amr_status upload(DevBuf<T> &b, const std::vector<T> &h, cudaStream_t s) {
    if (h.empty()) return AMR_OK;
    amr_status st = b.reserve(h.size());
    if (st) return st;
    return cuda_fail(cudaMemcpyAsync(b.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s), "h2d");
}

// Neighbour (gather) plan of a level from its host tables.
amr_status plan_level(amr_hydro_ctx *c, int level) {
    Level &L = c->lv[level];
    L.n_ghost = 0;
    if (!L.n_patches) return AMR_OK;
    int cells[3];
    for (int d = 0; d < 3; d++) cells[d] = c->prm.root_n[d] << level;
    std::vector<int32_t> nbr;
    std::vector<GhostInfo> ghosts;
    amr_status st = build_nbr_plan(level, L.n_patches, L.corner.data(), L.sib.data(),
                                   level > 0 ? L.parent.data() : nullptr, cells, nbr, ghosts,
                                   c->prm.recon == AMR_RECON_PPM ? 4 : 2, c->prm.fallback != 0);
    if (st) return st;
    if ((st = upload(L.nbr, nbr, c->stream))) return st;
    {  // z-runs of the length the round-robin cost estimate prefers
        std::vector<int32_t> chains, coff, runs, off;
        z_chains(L.n_groups, nbr.data(), chains, coff);
        const int len = choose_run_len(coff, c->n_sm * c->step_bps, c->prm.prec == AMR_FP64 ? 0.05 : 0.13);
        // single-group runs: the plain group list (a run list would only add
        // the lookups of each work item's group ahead of its tables)
        L.n_runs = 0;
        if (len > 1) {
            cut_runs(chains, coff, len, runs, off);
            L.n_runs = (int)off.size() - 1;
            if ((st = upload(L.runs, runs, c->stream)) || (st = upload(L.run_off, off, c->stream))) return st;
        }
    }
    L.n_ghost = (int)ghosts.size();
    if (L.n_ghost) {
        if ((st = L.ghost.reserve((size_t)L.n_ghost * PSLOT_H))) return st;
        std::vector<int32_t> gi((size_t)L.n_ghost * GHOST_INFO, 0);
        for (int i = 0; i < L.n_ghost; i++) {
            gi[GHOST_INFO * i] = ghosts[i].cparent;
            gi[GHOST_INFO * i + 1] = ghosts[i].qx;
            gi[GHOST_INFO * i + 2] = ghosts[i].qy;
            gi[GHOST_INFO * i + 3] = ghosts[i].qz;
            gi[GHOST_INFO * i + 4] = ghosts[i].box;
        }
        if ((st = upload(L.ghost_info, gi, c->stream))) return st;
    }
    return cuda_fail(cudaStreamSynchronize(c->stream), "sync");
}

// Coarse-fine registers between coarse level l-1 and fine level l, fix-up
// and restriction lists of the coarse level.  An interface is a face of a
// leaf coarse patch Q whose neighbour P across it is refined; the fine side
// is the face of P's child group toward Q.
amr_status rebuild_cf(amr_hydro_ctx *c, int l) {
    Level &C = c->lv[l - 1], &F = c->lv[l];
    C.n_creg = C.n_fix = C.n_restrict = 0;
    F.n_freg = 0;
    if (!C.n_patches || !F.n_patches) return AMR_OK;
    std::vector<int64_t> foff((size_t)F.n_groups * 6, -1), coff((size_t)C.n_patches * 6, -1), fix;
    std::vector<int32_t> rlist;
    int nf = 0, nc = 0;
    // fine side
    for (int g = 0; g < F.n_groups; g++) {
        const int P = F.parent[8 * g];
        if (P < 0 || P >= C.n_patches) return AMR_E_NESTING;
        for (int f = 0; f < 6; f++) {
            const int Q = C.sib[(size_t)P * 26 + face_sib(f)];
            if (Q < 0) return AMR_E_NESTING;
            if (C.child[Q] < 0) foff[(size_t)g * 6 + f] = (int64_t)(nf++) * 1280;
        }
    }
    // coarse side
    for (int Q = 0; Q < C.n_patches; Q++) {
        if (C.child[Q] >= 0) {
            rlist.push_back(Q);
            rlist.push_back(C.child[Q]);
            continue;
        }
        std::array<int64_t, 13> e;
        e.fill(-1);
        e[0] = Q;
        bool any = false;
        for (int f = 0; f < 6; f++) {
            const int P = C.sib[(size_t)Q * 26 + face_sib(f)];
            if (P < 0 || C.child[P] < 0) continue;
            const int G = C.child[P];
            const int64_t fo = foff[(size_t)G * 6 + (f ^ 1)];
            if (fo < 0) return AMR_E_NESTING;
            coff[(size_t)Q * 6 + f] = (int64_t)(nc++) * 320;
            e[1 + f] = coff[(size_t)Q * 6 + f];
            e[7 + f] = fo;
            any = true;
        }
        if (any) fix.insert(fix.end(), e.begin(), e.end());
    }
    amr_status st;
    if ((st = upload(F.fine_off, foff, c->stream))) return st;
    if ((st = upload(C.coarse_off, coff, c->stream))) return st;
    if ((st = upload(C.fix_list, fix, c->stream))) return st;
    if ((st = upload(C.restrict_list, rlist, c->stream))) return st;
    if (nf && (st = F.freg.reserve((size_t)nf * 1280))) return st;
    if (nc && (st = C.creg.reserve((size_t)nc * 320))) return st;
    if (nf && (st = cuda_fail(cudaMemsetAsync(F.freg.p, 0, sizeof(double) * 1280 * (size_t)nf, c->stream), "memset")))
        return st;
    F.n_freg = nf;
    C.n_creg = nc;
    C.n_fix = (int)(fix.size() / 13);
    C.n_restrict = (int)(rlist.size() / 2);
    return cuda_fail(cudaStreamSynchronize(c->stream), "sync");
}

}  // namespace amrh

using namespace amrh;

extern "C" {

amr_status amr_hydro_bind_level(amr_hydro_ctx *c, int level, double *U_a, double *U_b, int32_t *corner,
                                int32_t *sib, int32_t *parent, int32_t *child_group) {
    if (!c || level < 1 || level > c->prm.lmax) return AMR_E_INVAL;
    if (!U_a || !U_b || U_a == U_b || !corner || !sib || !parent || !child_group) return AMR_E_INVAL;
    Level &L = c->lv[level];
    L.bound = true;
    L.U[0] = U_a;
    L.U[1] = U_b;
    L.cur = 0;
    L.d_corner = L.w_corner = corner;
    L.d_sib = L.w_sib = sib;
    L.d_parent = L.w_parent = parent;
    L.d_child = L.w_child = child_group;
    L.n_patches = L.n_groups = 0;
    L.n_ghost = 0;
    L.corner.clear();
    L.sib.clear();
    L.parent.clear();
    L.child.clear();
    L.scal0 = SCAL_LEVEL0 + SCAL_PER * level;
    L.ring = 0;
    L.speed_valid = false;
    L.dt_prev = -1.0;
    return AMR_OK;
}

amr_status amr_hydro_level_info(amr_hydro_ctx *c, int level, int *n_patches, int *n_ghost) {
    if (!c || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    if (n_patches) *n_patches = c->lv[level].n_patches;
    if (n_ghost) *n_ghost = c->lv[level].n_ghost;
    return AMR_OK;
}

amr_status amr_hydro_regrid(amr_hydro_ctx *c, int l) {
    if (!c || l < 0 || l >= c->prm.lmax) return AMR_E_INVAL;
    Level &L = c->lv[l], &F = c->lv[l + 1];
    if (!L.n_patches || !F.bound) return AMR_E_INVAL;
    amr_status st;
    if ((st = level_time(c, l))) return st;
    const int n = L.n_patches;
    // device flags (cell criterion + flag buffer) -> host
    if ((st = c->pflag.reserve(n))) return st;
    if ((st = patch_flags_dev(c, l, c->pflag.p))) return st;
    std::vector<uint8_t> pflag(n);
    if ((st = cuda_fail(cudaMemcpyAsync(pflag.data(), c->pflag.p, n, cudaMemcpyDeviceToHost, c->stream), "d2h")))
        return st;
    if ((st = cuda_fail(cudaStreamSynchronize(c->stream), "sync"))) return st;

    int pc[3], fc[3];  // patches per dimension on levels l and l+1
    for (int d = 0; d < 3; d++) {
        pc[d] = (c->prm.root_n[d] << l) / 8;
        fc[d] = 2 * pc[d];
    }
    // patch position -> slot, dense over each level's patch grid
    std::vector<int32_t> at_l((size_t)pc[0] * pc[1] * pc[2], -1);
    auto idx_l = [&](int x, int y, int z) { return ((size_t)z * pc[1] + y) * pc[0] + x; };
    auto idx_f = [&](int x, int y, int z) { return ((size_t)z * fc[1] + y) * fc[0] + x; };
    for (int s = 0; s < n; s++) at_l[idx_l(L.corner[3 * s] / 8, L.corner[3 * s + 1] / 8, L.corner[3 * s + 2] / 8)] = s;

    // keep-for-nesting: level-l parents of the 27-neighbourhoods of refined
    // level-(l+1) patches stay refined
    std::vector<uint8_t> keep(n, 0);
    if (l + 2 <= c->prm.lmax && c->lv[l + 2].n_patches) {
        for (int x = 0; x < F.n_patches; x++) {
            if (F.child[x] < 0) continue;
            const int X[3] = {F.corner[3 * x] / 8, F.corner[3 * x + 1] / 8, F.corner[3 * x + 2] / 8};
            for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        const int q[3] = {wrapi(X[0] + dx, fc[0]) / 2, wrapi(X[1] + dy, fc[1]) / 2,
                                          wrapi(X[2] + dz, fc[2]) / 2};
                        const int32_t q_slot = at_l[idx_l(q[0], q[1], q[2])];
                        if (q_slot < 0) return AMR_E_NESTING;
                        keep[q_slot] = 1;
                    }
        }
    }
    // new refinement: flagged and properly nested, or kept
    std::vector<int> chosen;
    for (int s = 0; s < n; s++) {
        bool nest_ok = true;
        for (int k = 0; k < 26 && nest_ok; k++) nest_ok = L.sib[(size_t)s * 26 + k] >= 0;
        if ((pflag[s] && nest_ok) || (keep[s] && L.child[s] >= 0)) chosen.push_back(s);
    }
    // canonical group order: parents sorted by corner (z, y, x)
    std::sort(chosen.begin(), chosen.end(), [&](int a, int b) {
        for (int d = 2; d >= 0; d--)
            if (L.corner[3 * a + d] != L.corner[3 * b + d]) return L.corner[3 * a + d] < L.corner[3 * b + d];
        return a < b;
    });
    const int ng = (int)chosen.size(), nn = 8 * ng;
    // nothing to do when the refined set is unchanged: the existing groups
    // are already numbered in the canonical order of their parents
    if (ng == F.n_groups) {
        bool same = true;
        for (int g = 0; g < ng && same; g++) same = L.child[chosen[g]] == g;
        if (same) return AMR_OK;
    }
    if (nn > c->prm.max_patches) return AMR_E_NOMEM;

    std::vector<int32_t> corner((size_t)nn * 3), sib((size_t)nn * 26), parent(nn), child(nn, -1);
    std::vector<int32_t> old_of(nn, -1), new_of((size_t)F.n_patches, -1), lchild(n, -1), jobs, job_slot;
    std::vector<int32_t> at_f((size_t)fc[0] * fc[1] * fc[2], -1);
    for (int g = 0; g < ng; g++) {
        const int P = chosen[g];
        lchild[P] = g;
        for (int k = 0; k < 8; k++) {
            const int s = 8 * g + k, lx = k & 1, ly = (k >> 1) & 1, lz = k >> 2;
            corner[3 * s] = 2 * L.corner[3 * P] + 8 * lx;
            corner[3 * s + 1] = 2 * L.corner[3 * P + 1] + 8 * ly;
            corner[3 * s + 2] = 2 * L.corner[3 * P + 2] + 8 * lz;
            parent[s] = P;
            at_f[idx_f(corner[3 * s] / 8, corner[3 * s + 1] / 8, corner[3 * s + 2] / 8)] = s;
            if (L.child[P] >= 0) {
                const int o = 8 * L.child[P] + k;
                old_of[s] = o;
                new_of[o] = s;
                child[s] = F.child[o];
            } else {
                jobs.insert(jobs.end(), {P, lx, ly, lz, 8 << 12 | 8 << 16 | 8 << 20, 0, 0, 0});  // whole patch
                job_slot.push_back(s);
            }
        }
    }
    // sibling tables from each new group's 4x4x4 block of patch positions
    // (64 lookups per group instead of 26 per patch)
    auto wrapc = [](int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); };  // |step| <= 1 patch
    for (int g = 0; g < ng; g++) {
        int q[3][4];
        for (int d = 0; d < 3; d++) {
            const int b = corner[3 * (8 * g) + d] / 8;  // the group's low patch position
            for (int i = 0; i < 4; i++) q[d][i] = wrapc(b - 1 + i, fc[d]);
        }
        int32_t blk[64];
        for (int z = 0; z < 4; z++)
            for (int y = 0; y < 4; y++) {
                const size_t row = ((size_t)q[2][z] * fc[1] + q[1][y]) * fc[0];
                for (int x = 0; x < 4; x++) blk[x + 4 * y + 16 * z] = at_f[row + q[0][x]];
            }
        for (int k = 0; k < 8; k++) {
            const int lx = k & 1, ly = (k >> 1) & 1, lz = k >> 2;
            int32_t *o = &sib[(size_t)(8 * g + k) * 26];
            int m = 0;  // sibling index order: dx fastest, the patch itself skipped
            for (int dz = 0; dz < 3; dz++)
                for (int dy = 0; dy < 3; dy++)
                    for (int dx = 0; dx < 3; dx++)
                        if (dx != 1 || dy != 1 || dz != 1) o[m++] = blk[(lx + dx) + 4 * (ly + dy) + 16 * (lz + dz)];
        }
    }
    // grandchildren keep their data; their parent slots are renumbered
    Level *G2 = (l + 2 <= c->prm.lmax && c->lv[l + 2].n_patches) ? &c->lv[l + 2] : nullptr;
    std::vector<int32_t> g2parent;
    if (G2) {
        g2parent.resize(G2->n_patches);
        for (int y = 0; y < G2->n_patches; y++) {
            const int op = G2->parent[y];
            if (op < 0 || op >= (int)new_of.size() || new_of[op] < 0) return AMR_E_NESTING;
            g2parent[y] = new_of[op];
        }
    }

    // cell data of the new level l+1 into its other buffer
    const int dst = F.n_patches ? 1 - F.cur : 0;
    double *Ud = F.U[dst];
    const int ntmp = nn + (int)jobs.size() + (int)job_slot.size();
    if ((st = c->regrid_tmp.reserve(ntmp > 0 ? ntmp : 1))) return st;
    std::vector<int32_t> tmp;
    tmp.reserve(ntmp);
    tmp.insert(tmp.end(), old_of.begin(), old_of.end());
    tmp.insert(tmp.end(), jobs.begin(), jobs.end());
    tmp.insert(tmp.end(), job_slot.begin(), job_slot.end());
    if (!tmp.empty() &&
        (st = cuda_fail(cudaMemcpyAsync(c->regrid_tmp.p, tmp.data(), 4 * tmp.size(), cudaMemcpyHostToDevice, c->stream),
                        "h2d")))
        return st;
    if (F.n_patches && (st = copy_slots(c, Ud, F.U[F.cur], c->regrid_tmp.p, nn))) return st;
    if ((st = interp_new_patches(c, l, Ud, c->regrid_tmp.p + nn + jobs.size(), c->regrid_tmp.p + nn,
                                 (int)job_slot.size())))  // jobs: GHOST_INFO ints each
        return st;

    // tables: host mirrors and the caller's arrays
    F.corner = std::move(corner);
    F.sib = std::move(sib);
    F.parent = std::move(parent);
    F.child = std::move(child);
    F.n_patches = nn;
    F.n_groups = ng;
    F.cur = dst;
    F.t = F.t_prev = L.t;
    F.t_pending = false;
    F.speed_valid = false;
    F.ring = 0;
    L.child = std::move(lchild);
    auto put = [&](int32_t *d, const std::vector<int32_t> &h) -> amr_status {
        if (!d || h.empty()) return AMR_OK;
        return cuda_fail(cudaMemcpyAsync(d, h.data(), 4 * h.size(), cudaMemcpyHostToDevice, c->stream), "h2d");
    };
    if ((st = put(F.w_corner, F.corner)) || (st = put(F.w_sib, F.sib)) || (st = put(F.w_parent, F.parent)) ||
        (st = put(F.w_child, F.child)))
        return st;
    if ((st = put(L.w_child, L.child))) return st;
    if (G2) {
        G2->parent = std::move(g2parent);
        if ((st = put(G2->w_parent, G2->parent))) return st;
    }
    {
        const double rec[3] = {0.0, F.t, F.t};
        if ((st = cuda_fail(cudaMemcpyAsync(c->dtbuf.p + 3 * (l + 1), rec, 24, cudaMemcpyHostToDevice, c->stream),
                            "h2d time")))
            return st;
    }
    if ((st = cuda_fail(cudaMemsetAsync(c->scal.p + F.scal0, 0, 8 * SCAL_PER, c->stream), "memset"))) return st;
    if ((st = cuda_fail(cudaStreamSynchronize(c->stream), "sync"))) return st;
    if (!ng) F.dt_prev = -1.0;
    // plans of the changed levels
    if ((st = plan_level(c, l + 1))) return st;
    if ((st = rebuild_cf(c, l + 1))) return st;
    if (G2) {
        if ((st = plan_level(c, l + 2))) return st;
        if ((st = rebuild_cf(c, l + 2))) return st;
    }
    return AMR_OK;
}

}  // extern "C"

// ---- the W-cycle ------------------------------------------------------------------

namespace {

amr_status min_dt_host(amr_hydro_ctx *c, int l, double *dt) { return amr_hydro_min_dt(c, l, dt); }

// C_dec rule: shrink dt to twice the finer level's last step when that
// removes a small synchronisation step there.
double dec_rule(amr_hydro_ctx *c, int l, double dt) {
    if (l < c->prm.lmax && c->lv[l + 1].n_patches && c->lv[l + 1].dt_prev > 0.0) {
        const double d2 = 2.0 * c->lv[l + 1].dt_prev;
        if (dt > d2 && (1.0 - c->prm.c_dec) * dt < d2) return d2;
    }
    return dt;
}

amr_status advance_rec(amr_hydro_ctx *c, int l, double dt0, int64_t *updates) {
    Level &L = c->lv[l];
    amr_status st;
    double target, dt = 0.0;
    if (l == 0) {
        dt = dt0;
        if (!(dt > 0.0) && (st = min_dt_host(c, 0, &dt))) return st;
        dt = dec_rule(c, 0, dt);
        target = L.t + dt;
    } else {
        target = c->lv[l - 1].t;
    }
    while (L.t < target) {
        bool last = false;
        double step;
        if (l == 0) {
            step = dt;
        } else {
            if ((st = min_dt_host(c, l, &step))) return st;
            if ((1.0 + c->prm.c_inc) * step > target - L.t) {
                step = target - L.t;
                last = true;
            } else {
                step = dec_rule(c, l, step);
            }
        }
        if ((st = amr_hydro_advance_level(c, l, step, nullptr))) return st;
        if (L.dt_last != step) {  // the level retried with a smaller dt (remedy iv)
            step = L.dt_last;
            last = false;
            if (l == 0) target = L.t;
        }
        if (last || l == 0) L.t = target;
        L.dt_prev = step;
        if (updates) *updates += (int64_t)L.n_patches * 512;
        if (l < c->prm.lmax && c->lv[l + 1].n_patches) {
            if ((st = advance_rec(c, l + 1, 0.0, updates))) return st;
            if ((st = amr_hydro_flux_fixup(c, l))) return st;
        }
        if (l < c->prm.lmax && c->lv[l + 1].bound) {
            if ((st = amr_hydro_regrid(c, l))) return st;
        }
    }
    return AMR_OK;
}

}  // namespace

extern "C" amr_status amr_hydro_advance_root(amr_hydro_ctx *c, double dt0, int64_t *cell_updates) {
    if (!c || !c->lv[0].n_patches) return AMR_E_INVAL;
    if (cell_updates) *cell_updates = 0;
    return advance_rec(c, 0, dt0, cell_updates);
}
