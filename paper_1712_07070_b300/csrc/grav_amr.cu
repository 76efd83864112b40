// grav_amr.cu -- self-gravity inside the adaptive time-step W-cycle (GAMER-2
// section 2.3 on the section 2.1 hierarchy).
//
// Every level keeps its potential and acceleration at its newest time
// (buffers gc) and at its previous time (1 - gc).  A level step from t to
// t + dt:
//   * g^n of the coarse-fine ghost patches, interpolated from the coarse
//     level's accelerations (time, then the minmod-limited prolongation);
//   * the predictor: the step kernel's MUSCL-Hancock instance with
//     (dt/2)(0, rho g, m.g) in its half step;
//   * the potential of the predicted density at t + dt: the root's periodic
//     FFT solve, or a refined level's per-patch 18^3 SOR with the parent's
//     potential interpolated linearly in time (w clamped to [0, 1]; 1 when
//     the parent holds a single time) -- one Poisson solve per level step;
//   * the corrector with g^n and g^{n+1}, which also reduces the next CFL
//     signal speed.
// A regrid that changes a level solves its potential again at its time.
#include <cuda_runtime.h>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

namespace amrh {

// The parent's time weight for a solve of level l at time t.
static double parent_weight(const Level &C, double t) {
    if (C.t == C.t_prev || t >= C.t) return 1.0;
    const double w = (t - C.t_prev) / (C.t - C.t_prev);
    return w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
}

// Potential and acceleration of `level` at its newest time into its buffers
// 1 - gc (the step's predicted state, or the state a regrid left).
static amr_status solve_into(amr_hydro_ctx *c, int level, int slot, double t) {
    Level &L = c->lv[level];
    if (!L.n_patches) return AMR_OK;
    const size_t n = (size_t)L.n_patches * PV;
    amr_status st;
    if ((st = L.phi[slot].reserve(level ? (size_t)c->prm.max_patches * PV : n)) ||
        (st = L.gacc[slot].reserve(level ? (size_t)c->prm.max_patches * 3 * PV : 3 * n)))
        return st;
    if (level == 0) return amr_hydro_poisson_root(c, c->grav_G, L.phi[slot].p, L.gacc[slot].p, c->grav_order);
    Level &C = c->lv[level - 1];
    if ((st = level_time(c, level - 1))) return st;
    return amr_hydro_poisson_level_t(c, level, c->grav_G, c->grav_omega, c->grav_iters, C.phi[1 - C.gc].p,
                                     C.phi[C.gc].p, parent_weight(C, t), L.phi[slot].p, L.gacc[slot].p,
                                     c->grav_order);
}

// The level's potential and acceleration at its current time, in both of
// its buffers (initially, and after a regrid changed the level).
amr_status gravity_solve_level(amr_hydro_ctx *c, int level) {
    Level &L = c->lv[level];
    if (!L.n_patches) return AMR_OK;
    amr_status st;
    if ((st = level_time(c, level))) return st;
    L.gc = 0;
    if ((st = solve_into(c, level, 0, L.t))) return st;
    const size_t n = (size_t)L.n_patches * PV;
    if ((st = L.phi[1].reserve(L.phi[0].cap)) || (st = L.gacc[1].reserve(L.gacc[0].cap))) return st;
    if ((st = cuda_fail(cudaMemcpyAsync(L.phi[1].p, L.phi[0].p, 8 * n, cudaMemcpyDeviceToDevice, c->stream),
                        "d2d")) ||
        (st = cuda_fail(cudaMemcpyAsync(L.gacc[1].p, L.gacc[0].p, 24 * n, cudaMemcpyDeviceToDevice, c->stream),
                        "d2d")))
        return st;
    return AMR_OK;
}

// One coupled step of a level inside the W-cycle (host dt).
amr_status gravity_level_step(amr_hydro_ctx *c, int level, double dt) {
    Level &L = c->lv[level];
    amr_status st;
    if ((st = level_time(c, level))) return st;
    if (L.n_ghost && (st = fill_ghost_acc(c, level, L.t))) return st;
    const int gc = L.gc;
    const double *acc_n = L.gacc[gc].p;
    if ((st = advance_once(c, level, dt, nullptr, acc_n))) return st;  // the predictor
    if ((st = solve_into(c, level, 1 - gc, L.t))) return st;             // at t + dt
    if ((st = launch_grav_correct(c, level, dt, acc_n, L.gacc[1 - gc].p))) return st;
    L.gc = 1 - gc;
    return AMR_OK;
}

}  // namespace amrh

using namespace amrh;

extern "C" {

amr_status amr_hydro_set_gravity(amr_hydro_ctx *c, double G, double omega, int iters, int acc_order) {
    if (!c || !(G >= 0.0) || !(omega > 0.0 && omega < 2.0) || iters < 0 || (acc_order != 2 && acc_order != 4))
        return AMR_E_INVAL;
    // the coupling is built for MUSCL-Hancock + PLM without dual energy, the
    // remedies or the level retry, on periodic roots
    if (c->prm.scheme != AMR_SCHEME_MH || c->prm.recon != AMR_RECON_PLM || c->prm.dual_energy ||
        c->prm.fallback || c->prm.dt_min > 0.0 || c->prm.gravity_bc != AMR_GRAVITY_PERIODIC)
        return AMR_E_INVAL;
    if (!c->lv[0].n_patches) return AMR_E_INVAL;
    c->grav_G = G;
    c->grav_omega = omega;
    c->grav_iters = iters;
    c->grav_order = acc_order;
    c->grav_on = true;
    amr_status st;
    for (int l = 0; l <= c->prm.lmax; l++)
        if ((st = gravity_solve_level(c, l))) return st;
    return AMR_OK;
}

amr_status amr_hydro_level_gravity(amr_hydro_ctx *c, int level, double *phi_out, double *acc_out) {
    if (!c || level < 0 || level > c->prm.lmax || !c->grav_on) return AMR_E_INVAL;
    Level &L = c->lv[level];
    const size_t n = (size_t)L.n_patches * PV;
    if (!n) return AMR_OK;
    amr_status st;
    if (phi_out && (st = cuda_fail(cudaMemcpyAsync(phi_out, L.phi[L.gc].p, 8 * n, cudaMemcpyDeviceToDevice,
                                                   c->stream), "d2d")))
        return st;
    if (acc_out && (st = cuda_fail(cudaMemcpyAsync(acc_out, L.gacc[L.gc].p, 24 * n, cudaMemcpyDeviceToDevice,
                                                   c->stream), "d2d")))
        return st;
    return cuda_fail(cudaStreamSynchronize(c->stream), "sync");
}

}  // extern "C"
