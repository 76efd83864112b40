// regrid.cpp -- the host side of the AMR bookkeeping (GAMER-2 section 2.1):
//   * gather plans and coarse-fine register maps of levels registered from
//     host tables (amr_hydro_set_level);
//   * the regrid entry point (the work runs on the device, regrid_dev.cu);
//   * the adaptive time-step W-cycle with the C_inc / C_dec rule of the
//     section's pseudo-code, followed by fix-up (section 2.2) and regrid.
#include <cuda_runtime.h>

#include <array>
#include <cstring>
#include <vector>

#include "amr_hydro.h"
#include "ctx.h"

namespace amrh {

constexpr int PSLOT_H = 5 * 512;

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
    L.plan_version++;
    L.ghost_valid = false;
    L.n_runs = 0;
    L.has_work = false;  // the host tables' group order is the caller's
    if (!L.n_patches) return AMR_OK;
    amr_status st0 = refresh_host_tables(c, level);
    if (st0) return st0;
    int cells[3];
    for (int d = 0; d < 3; d++) cells[d] = c->prm.root_n[d] << level;
    std::vector<int32_t> nbr;
    std::vector<GhostInfo> ghosts;
    amr_status st = build_nbr_plan(level, L.n_patches, L.corner.data(), L.sib.data(),
                                   level > 0 ? L.parent.data() : nullptr, cells, nbr, ghosts,
                                   (c->prm.recon == AMR_RECON_PPM || c->prm.scheme == AMR_SCHEME_VL) ? 4 : 2,
                                   c->prm.fallback != 0);
    if (st) return st;
    if ((st = upload(L.nbr, nbr, c->stream))) return st;
    {  // z-runs of the length the round-robin cost estimate prefers
        std::vector<int32_t> chains, coff, runs, off;
        z_chains(L.n_groups, nbr.data(), chains, coff);
        const int len = choose_run_len(coff, c->n_sm * c->step_bps, c->prm.prec == AMR_FP64 ? 0.05 : 0.13);
        // single-group runs: the plain group list (a run list would only add
        // the lookups of each work item's group ahead of its tables)
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
    {
        const amr_status s0 = refresh_host_tables(c, l - 1);
        if (s0) return s0;
        const amr_status s1 = refresh_host_tables(c, l);
        if (s1) return s1;
    }
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
            if (C.child[Q] < 0) foff[(size_t)g * 6 + f] = (int64_t)(nf++) * fine_block(c);
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
            coff[(size_t)Q * 6 + f] = (int64_t)(nc++) * coarse_block(c);
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
    if (nf && (st = F.freg.reserve((size_t)nf * fine_block(c)))) return st;
    if (nc && (st = C.creg.reserve((size_t)nc * coarse_block(c)))) return st;
    if (nf && (st = cuda_fail(cudaMemsetAsync(F.freg.p, 0, sizeof(double) * fine_block(c) * (size_t)nf, c->stream),
                              "memset")))
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
    L.posmap_valid = L.ghost_valid = L.host_stale = false;
    L.has_work = false;
    L.n_runs = 0;
    L.version++;
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
    if ((st = level_time(c, l))) return st;  // the new children start at the level's time
    return regrid_dev(c, l);
}

}  // extern "C"

// ---- the W-cycle ------------------------------------------------------------------

namespace {

amr_status min_dt_host(amr_hydro_ctx *c, int l, double *dt) {
    PhaseScope ph(c, AMR_PH_DT);
    return amr_hydro_min_dt(c, l, dt);
}

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
        if (c->shared_dt) {  // the constraint of every level, the minimum
            if (!(dt > 0.0)) {
                if ((st = min_dt_host(c, 0, &dt))) return st;
                for (int k = 1; k <= c->prm.lmax; k++) {
                    if (!c->lv[k].n_patches) continue;
                    double dk;
                    if ((st = min_dt_host(c, k, &dk))) return st;
                    dt = dk < dt ? dk : dt;
                }
            }
            c->shared_step = dt;
        } else {
            if (!(dt > 0.0) && (st = min_dt_host(c, 0, &dt))) return st;
            dt = dec_rule(c, 0, dt);
        }
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
            // shared: the root step's dt, which lands on the parent's time
            if (c->shared_dt) step = c->shared_step;
            else if ((st = min_dt_host(c, l, &step))) return st;
            if ((1.0 + c->prm.c_inc) * step > target - L.t) {
                step = target - L.t;
                last = true;
            } else if (!c->shared_dt) {
                step = dec_rule(c, l, step);
            }
        }
        // with self-gravity the coupled step (predictor, the level's Poisson
        // solve at the step's end, corrector)
        if ((st = c->grav_on ? gravity_level_step(c, l, step) : amr_hydro_advance_level(c, l, step, nullptr)))
            return st;
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
            PhaseScope ph(c, AMR_PH_FIXUP);
            if ((st = amr_hydro_flux_fixup(c, l))) return st;
        }
        if (l < c->prm.lmax && c->lv[l + 1].bound) {
            PhaseScope ph(c, AMR_PH_REGRID);
            const unsigned long long before = c->lv[l + 1].structure;
            if ((st = amr_hydro_regrid(c, l))) return st;
            // a changed level solves its potential again at its time
            if (c->grav_on && c->lv[l + 1].structure != before && (st = gravity_solve_level(c, l + 1))) return st;
        }
    }
    return AMR_OK;
}

}  // namespace

extern "C" amr_status amr_hydro_set_shared_dt(amr_hydro_ctx *c, int on) {
    if (!c) return AMR_E_INVAL;
    c->shared_dt = on != 0;
    return AMR_OK;
}

extern "C" amr_status amr_hydro_advance_root(amr_hydro_ctx *c, double dt0, int64_t *cell_updates) {
    if (!c || !c->lv[0].n_patches) return AMR_E_INVAL;
    if (cell_updates) *cell_updates = 0;
    return advance_rec(c, 0, dt0, cell_updates);
}
