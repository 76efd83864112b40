// level.cu -- per-level entry points: registration of a level's arrays and
// the advance of all its patch groups by one step (GAMER-2 sections 2.1-2.2).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

using namespace amrh;

namespace amrh {

// Bring a level's host-side time up to date after device-side time steps.
static amr_status sync_level_time(amr_hydro_ctx *c, Level &L, int level) {
    if (!L.t_pending) return AMR_OK;
    double rec[3];
    amr_status st = cuda_fail(cudaMemcpyAsync(rec, c->dtbuf.p + 3 * level, 24, cudaMemcpyDeviceToHost,
                                              c->stream), "d2h time");
    if (st) return st;
    if ((st = cuda_fail(cudaStreamSynchronize(c->stream), "sync"))) return st;
    L.t = rec[1];
    L.t_prev = rec[2];
    L.t_pending = false;
    return AMR_OK;
}

}  // namespace amrh

extern "C" {

amr_status amr_hydro_set_level(amr_hydro_ctx *c, int level, int n_patches, double *U_a, double *U_b,
                               const int32_t *corner, const int32_t *sib, const int32_t *parent,
                               int32_t *child_group, double t) {
    if (!c || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    if (n_patches < 0 || n_patches % 8 || n_patches > c->prm.max_patches) return AMR_E_INVAL;
    if (n_patches > 0 && (!U_a || !U_b || !corner || !sib)) return AMR_E_INVAL;
    if (level > 0 && n_patches > 0 && !parent) return AMR_E_INVAL;
    // VL on a refined level needs the ghost-patch neighbour tables the
    // device-side regrid builds: refined levels come from amr_hydro_regrid
    if (level > 0 && n_patches > 0 && c->prm.scheme == AMR_SCHEME_VL) return AMR_E_INVAL;
    Level &L = c->lv[level];
    amr_status st;
    if ((st = cuda_fail(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize(), "sync")))
        return st;
    L.n_patches = n_patches;
    L.n_groups = n_patches / 8;
    L.U[0] = U_a;
    L.U[1] = U_b;
    L.S[0] = L.S[1] = nullptr;  // entropy fields: registered again after set_level
    L.cur = 0;
    L.t = L.t_prev = t;
    L.t_pending = false;
    L.d_corner = corner;
    L.d_sib = sib;
    L.d_parent = parent;
    L.d_child = child_group;
    L.w_child = child_group;
    L.scal0 = SCAL_LEVEL0 + SCAL_PER * level;
    L.ring = 0;
    L.speed_valid = false;
    L.posmap_valid = false;
    L.host_stale = false;
    L.ghost_valid = false;
    L.version++;
    if ((st = cuda_fail(cudaMemset(c->scal.p + L.scal0, 0, 8 * SCAL_PER), "memset"))) return st;
    L.n_ghost = 0;
    {
        const double rec[3] = {0.0, t, t};
        if ((st = cuda_fail(cudaMemcpy(c->dtbuf.p + 3 * level, rec, 24, cudaMemcpyHostToDevice), "h2d time")))
            return st;
    }
    if (n_patches == 0) return AMR_OK;

    L.corner.resize((size_t)n_patches * 3);
    L.sib.resize((size_t)n_patches * 26);
    L.parent.assign(n_patches, -1);
    L.child.assign(n_patches, -1);
    if ((st = cuda_fail(cudaMemcpy(L.corner.data(), corner, 12ull * n_patches, cudaMemcpyDeviceToHost), "d2h")))
        return st;
    if ((st = cuda_fail(cudaMemcpy(L.sib.data(), sib, 104ull * n_patches, cudaMemcpyDeviceToHost), "d2h")))
        return st;
    if (parent && (st = cuda_fail(cudaMemcpy(L.parent.data(), parent, 4ull * n_patches, cudaMemcpyDeviceToHost), "d2h")))
        return st;
    if (child_group && (st = cuda_fail(cudaMemcpy(L.child.data(), child_group, 4ull * n_patches, cudaMemcpyDeviceToHost), "d2h")))
        return st;

    int cells[3];
    for (int d = 0; d < 3; d++) cells[d] = c->prm.root_n[d] << level;
    for (int i = 0; i < 3 * n_patches; i++)
        if (L.corner[i] < 0 || L.corner[i] >= cells[i % 3] || L.corner[i] % 8) return AMR_E_INVAL;
    // the whole root grid in the slot order of amr_hydro_uniform_tables
    // (groups x-fastest, patches x-fastest within a group)?
    L.uniform = false;
    if (level == 0 && (int64_t)n_patches * 512 == (int64_t)cells[0] * cells[1] * cells[2]) {
        const int ngx = cells[0] / 16, ngy = cells[1] / 16;
        bool ok = cells[0] % 16 == 0 && cells[1] % 16 == 0 && cells[2] % 16 == 0;
        for (int s = 0; s < n_patches && ok; s++) {
            const int g = s / 8, k = s % 8;
            ok = L.corner[3 * s] == 16 * (g % ngx) + 8 * (k & 1) &&
                 L.corner[3 * s + 1] == 16 * ((g / ngx) % ngy) + 8 * ((k >> 1) & 1) &&
                 L.corner[3 * s + 2] == 16 * (g / (ngx * ngy)) + 8 * (k >> 2);
        }
        L.uniform = ok;
    }
    if (c->prm.scheme == AMR_SCHEME_VL && (st = L.ustar.reserve((size_t)n_patches * PSLOT))) return st;
    if ((st = plan_level(c, level))) return st;
    if (level > 0 && (st = rebuild_cf(c, level))) return st;
    if (level < c->prm.lmax && c->lv[level + 1].n_patches && (st = rebuild_cf(c, level + 1))) return st;
    return AMR_OK;
}

amr_status amr_hydro_set_entropy(amr_hydro_ctx *c, int level, double *S_a, double *S_b) {
    if (!c || level < 0 || level > c->prm.lmax || !c->prm.dual_energy) return AMR_E_INVAL;
    Level &L = c->lv[level];
    // a level with patches, or a refined level's capacity arrays (bind_level)
    if ((!L.n_patches && !L.bound) || !S_a || !S_b || S_a == S_b) return AMR_E_INVAL;
    L.S[L.cur] = S_a;
    L.S[1 - L.cur] = S_b;
    return AMR_OK;
}

amr_status amr_hydro_touch_level(amr_hydro_ctx *c, int level) {
    if (!c || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    Level &L = c->lv[level];
    if (!L.n_patches) return AMR_E_INVAL;
    L.speed_valid = false;
    L.version++;
    return AMR_OK;
}

}  // extern "C"

namespace amrh {

// The launches of one level step on c->stream: the fine registers' reset,
// the step launch(es) and the cell remedies (P: the step's parameters).
static amr_status launch_level_step(amr_hydro_ctx *c, int level, StepParams &P, const double *acc_n) {
    Level &L = c->lv[level];
    amr_status st;
    if (level < c->prm.lmax) {  // a coarse step restarts the fine level's flux sums
        Level &F = c->lv[level + 1];
        if (F.n_patches && F.n_freg &&
            (st = cuda_fail(cudaMemsetAsync(F.freg.p, 0, sizeof(double) * fine_block(c) * (size_t)F.n_freg, c->stream),
                            "memset fine registers")))
            return st;
    }
    if (L.n_runs > 0) {  // z-runs of groups as the work items
        P.runs = L.runs.p;
        P.run_off = L.run_off.p;
        P.n_work = L.n_runs;
    } else if (L.has_work) {  // single groups in position order (neighbours share ghost reads in L2)
        P.work = L.work.p;
    }
    const int cap = c->n_sm * c->step_bps;
    const int grid = P.n_work < cap ? P.n_work : cap;
    {
        int lo, hi;
        scheme_stages(c->prm.scheme, c->prm.recon, c->prm.dual_energy, lo, hi);
        P.stage = lo;  // MUSCL-Hancock (PLM, PPM, dual energy) or CTU: the one launch
        if (acc_n) {  // the gravity coupling's predictor
            P.stage = c->prm.scheme == AMR_SCHEME_CTU ? ST_CTU_GRAV : ST_MH_GRAV;
            P.acc_n = acc_n;
            P.ghost_acc = L.n_ghost ? L.ghost_acc.p : nullptr;
        }
    }
    if (c->prm.scheme == AMR_SCHEME_VL) {  // predictor into U*, then the corrector
        StepParams H = P;
        H.stage = ST_VL_PRED;
        H.U_new = L.ustar.p;
        H.smax_out = H.n_bad = H.clear2 = nullptr;
        H.time_rec = nullptr;
        H.cf = CFRegs{nullptr, nullptr, nullptr, nullptr};
        H.fb_count = nullptr;
        H.fb_list = nullptr;
        if ((st = launch_step(c, H, grid))) return st;
        // refined levels: the half step of the ghost cells the corrector reads
        if (L.n_ghost && (st = launch_vl_ghost_pred(c, level, H))) return st;
        P.stage = ST_VL_CORR;
        P.U_base = P.U_old;
        P.U_old = L.ustar.p;
        if (L.n_ghost) P.ghost = L.ghost_ustar.p;
    }
    if ((st = launch_step(c, P, grid))) return st;
    {
        StepParams R = P;  // the cell remedies recompute from U^n: its ghosts
        R.ghost = L.ghost.p;
        if ((st = launch_cell_remedies(c, R, P.stage == ST_VL_CORR ? P.U_base : P.U_old, stage_ctu(P.stage),
                                       c->stream)))
            return st;
    }

    return AMR_OK;
}

// One step of a level (the body of amr_hydro_advance_level without the
// retry of remedy (iv)); acc_n: the gravity predictor's acceleration at t^n
// (null: no gravity); c_acc > 0 with dt < 0: dt also obeys Eq. (acc) on acc_n.
amr_status advance_once(amr_hydro_ctx *c, int level, double dt, int64_t *n_unphysical_out, const double *acc_n,
                        double c_acc) {
    Level &L = c->lv[level];
    amr_status st;
    if (L.n_ghost) {  // coarse-fine ghosts need the level's time on the host
        PhaseScope ph(c, AMR_PH_GHOST);
        if ((st = sync_level_time(c, L, level))) return st;
        if ((st = fill_ghost_impl(c, level, L.t))) return st;
    }
    PhaseScope ph_step(c, AMR_PH_STEP);
    if (dt < 0.0 && (st = level_speed(c, level))) return st;
    if (dt < 0.0 && acc_n && c_acc > 0.0 &&  // Eq. (acc) joins Eq. (CFL2)
        (st = launch_acc_speed(c, acc_n, (int64_t)L.n_patches * 3 * PV, level_dh(c, level), c_acc,
                               c->scal.p + L.scal0 + L.ring)))
        return st;
    unsigned long long *sc = c->scal.p + L.scal0;
    const int r_in = L.ring, r_out = (L.ring + 1) % 3, r_clr = (L.ring + 2) % 3;

    StepParams P;
    std::memset(&P, 0, sizeof(P));
    P.U_old = L.U[L.cur];
    P.U_new = L.U[1 - L.cur];
    P.nbr = L.nbr.p;
    P.ghost = L.ghost.p;
    P.work = nullptr;
    P.n_work = L.n_groups;
    P.dt = dt;
    P.smax_in = sc + r_in;
    P.cfl = c->prm.cfl;
    P.dh = level_dh(c, level);
    P.gamma = c->prm.gamma;
    P.limiter = c->prm.limiter;
    P.riemann = c->prm.riemann;
    P.theta = c->prm.minmod_coeff;
    P.fallback = c->prm.fallback;
    if (c->prm.dual_energy) {
        if (!L.S[0] || !L.S[1]) return AMR_E_INVAL;  // amr_hydro_set_entropy first
        P.S_old = L.S[L.cur];
        P.S_new = L.S[1 - L.cur];
        P.ghost_S = L.ghost_S.p;
        P.de_xi = c->prm.dual_xi;
    }
    if (c->prm.fallback) {
        P.fb_count = c->fb_count.p;
        P.fb_list = c->fb_list.p;
        P.fb_cap = FB_CAP;
    }
    P.smax_out = sc + r_out;
    P.n_bad = sc + 3 + r_out;
    P.clear2 = sc + r_clr;
    P.time_rec = c->dtbuf.p + 3 * level;
    P.cf.fine_off = L.n_freg ? L.fine_off.p : nullptr;
    P.cf.fine_buf = L.freg.p;
    P.cf.coarse_off = L.n_creg ? L.coarse_off.p : nullptr;
    P.cf.coarse_buf = L.creg.p;
    // On a refined hierarchy the launches of the level step (the fine
    // registers' reset, the persistent step launch over all the level's
    // groups -- two with VL, plus the ghost half step -- and the cell
    // remedies) are captured into one CUDA graph per level: each step's
    // capture updates the level's instantiated graph in place
    // (cudaGraphExecUpdate: same nodes, new parameters, also after a regrid)
    // and the graph runs on the context's stream.
    const bool as_graph = c->prm.lmax > 0;
    cudaStream_t stream0 = c->stream;
    if (as_graph) {
        if (!c->capture_stream &&
            (st = cuda_fail(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "stream")))
            return st;
        if ((st = cuda_fail(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal), "capture")))
            return st;
        c->stream = c->capture_stream;
    }
    st = launch_level_step(c, level, P, acc_n);
    if (as_graph) {
        c->stream = stream0;
        cudaGraph_t gr = nullptr;
        const amr_status ce = cuda_fail(cudaStreamEndCapture(c->capture_stream, &gr), "end capture");
        if (!st) st = ce;
        if (!st && L.gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(L.gexec, gr, &info) != cudaSuccess) {  // the nodes changed
                cudaGetLastError();
                cudaGraphExecDestroy(L.gexec);
                L.gexec = nullptr;
            }
        }
        if (!st && !L.gexec) st = cuda_fail(cudaGraphInstantiate(&L.gexec, gr, 0), "instantiate");
        if (gr) cudaGraphDestroy(gr);
        if (!st) st = cuda_fail(cudaGraphLaunch(L.gexec, c->stream), "graph launch");
    }
    if (st) return st;

    L.cur = 1 - L.cur;
    L.version++;
    if (dt >= 0.0 && !L.t_pending) {
        L.t_prev = L.t;
        L.t += dt;
    } else {
        L.t_pending = true;
    }
    L.ring = r_out;
    L.speed_valid = true;
    L.dt_last = dt;

    if (n_unphysical_out) {
        unsigned long long nb = 0;
        if ((st = cuda_fail(cudaMemcpyAsync(&nb, sc + 3 + r_out, 8, cudaMemcpyDeviceToHost, c->stream), "d2h")))
            return st;
        if ((st = cuda_fail(cudaStreamSynchronize(c->stream), "sync"))) return st;
        *n_unphysical_out = (int64_t)nb;
        if (nb) return AMR_E_UNPHYSICAL;
    }
    return AMR_OK;
}

}  // namespace amrh

extern "C" {

amr_status amr_hydro_advance_level(amr_hydro_ctx *c, int level, double dt, int64_t *n_unphysical_out) {
    if (!c || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    Level &L = c->lv[level];
    if (!L.n_patches) return AMR_E_INVAL;
    if (!(dt >= 0.0) && !(dt < 0.0)) return AMR_E_INVAL;  // NaN
    if (!(c->prm.dt_min > 0.0)) return advance_once(c, level, dt, n_unphysical_out, nullptr);

    // Remedies (iv)-(v) (section 2.2): while cells stay unphysical after the
    // per-cell remedies, recompute the whole level from U^n with dt x 0.8,
    // down to dt_min.  U^n is untouched by a step (it writes the other
    // buffer); the level's host time, ring position and device time record,
    // the reduction slots the step accumulated into and the fine flux
    // registers the step added to are put back before each retry.
    amr_status st;
    if ((st = sync_level_time(c, L, level))) return st;
    const int cur = L.cur, ring = L.ring;
    const bool valid = L.speed_valid;
    const double t = L.t, t_prev = L.t_prev;
    double rec[3];
    if ((st = cuda_fail(cudaMemcpy(rec, c->dtbuf.p + 3 * level, 24, cudaMemcpyDeviceToHost), "d2h time"))) return st;
    const size_t nfr = (size_t)fine_block(c) * L.n_freg;
    if (level > 0 && nfr) {
        if ((st = L.freg_save.reserve(nfr))) return st;
        if ((st = cuda_fail(cudaMemcpyAsync(L.freg_save.p, L.freg.p, 8 * nfr, cudaMemcpyDeviceToDevice, c->stream),
                            "save registers")))
            return st;
    }
    double step = dt;
    for (;;) {
        int64_t nb = 0;
        st = advance_once(c, level, step, &nb, nullptr);
        if (st != AMR_E_UNPHYSICAL) {
            if (n_unphysical_out) *n_unphysical_out = st == AMR_OK ? 0 : nb;
            return st;
        }
        if (step < 0.0) {  // the device took its own CFL dt
            double used[3];
            if ((st = cuda_fail(cudaMemcpy(used, c->dtbuf.p + 3 * level, 24, cudaMemcpyDeviceToHost), "d2h time")))
                return st;
            step = used[0];
        }
        L.cur = cur;
        L.ring = ring;
        L.speed_valid = valid;
        L.t = t;
        L.t_prev = t_prev;
        L.t_pending = false;
        unsigned long long *sc = c->scal.p + L.scal0;
        const int r_out = (ring + 1) % 3;
        if ((st = cuda_fail(cudaMemsetAsync(sc + r_out, 0, 8, c->stream), "memset")) ||
            (st = cuda_fail(cudaMemsetAsync(sc + 3 + r_out, 0, 8, c->stream), "memset")) ||
            (st = cuda_fail(cudaMemcpyAsync(c->dtbuf.p + 3 * level, rec, 24, cudaMemcpyHostToDevice, c->stream),
                            "h2d time")))
            return st;
        if (level > 0 && nfr &&
            (st = cuda_fail(cudaMemcpyAsync(L.freg.p, L.freg_save.p, 8 * nfr, cudaMemcpyDeviceToDevice, c->stream),
                            "restore registers")))
            return st;
        step *= 0.8;
        if (step < c->prm.dt_min) {
            if (n_unphysical_out) *n_unphysical_out = nb;
            return AMR_E_UNPHYSICAL;
        }
    }
}

}  // extern "C"

namespace amrh {
amr_status level_time(amr_hydro_ctx *c, int level) { return sync_level_time(c, c->lv[level], level); }
}  // namespace amrh
