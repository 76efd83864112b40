// amr_ops.cu -- coarse-fine operations of the AMR hierarchy (GAMER-2
// sections 2.1-2.2, 3.2): ghost interpolation, flux fix-up, restriction,
// refinement flags, conservation sums.
#include <cuda_runtime.h>

#include "amr_hydro.h"
#include "ctx.h"

using namespace amrh;

namespace amrh {
amr_status fill_ghost_impl(amr_hydro_ctx *c, int level, double t) {
    (void)c; (void)level; (void)t;
    return AMR_E_INVAL;
}
}  // namespace amrh

extern "C" {
amr_status amr_hydro_fill_ghost(amr_hydro_ctx *c, int level, double t) {
    if (!c || level <= 0 || level > c->prm.lmax) return AMR_E_INVAL;
    return fill_ghost_impl(c, level, t);
}
amr_status amr_hydro_flux_fixup(amr_hydro_ctx *c, int coarse_level) {
    (void)c; (void)coarse_level;
    return AMR_E_INVAL;
}
amr_status amr_hydro_regrid_flags(amr_hydro_ctx *c, int level, uint8_t *flags) {
    (void)c; (void)level; (void)flags;
    return AMR_E_INVAL;
}
amr_status amr_hydro_conserved_sum(amr_hydro_ctx *c, int level, double *out) {
    (void)c; (void)level; (void)out;
    return AMR_E_INVAL;
}
amr_status amr_hydro_set_box(amr_hydro_ctx *c, int box_id, int n, double *U_a, double *U_b) {
    (void)c; (void)box_id; (void)n; (void)U_a; (void)U_b;
    return AMR_E_INVAL;
}
amr_status amr_hydro_advance_boxes(amr_hydro_ctx *c, int n_boxes, const int *box_ids, int n_steps,
                                   double *dt_log) {
    (void)c; (void)n_boxes; (void)box_ids; (void)n_steps; (void)dt_log;
    return AMR_E_INVAL;
}
amr_status amr_hydro_box_state(amr_hydro_ctx *c, int box_id, int *cur) {
    (void)c; (void)box_id; (void)cur;
    return AMR_E_INVAL;
}
amr_status amr_hydro_step_adjoint(amr_hydro_ctx *c, int level, double dt, const double *U_n,
                                  const double *lam_np1, double *lam_n) {
    (void)c; (void)level; (void)dt; (void)U_n; (void)lam_np1; (void)lam_n;
    return AMR_E_INVAL;
}
}
