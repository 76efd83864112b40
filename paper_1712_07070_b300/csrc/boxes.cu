// boxes.cu -- independent periodic boxes advanced together.
#include <cuda_runtime.h>

#include "amr_hydro.h"
#include "ctx.h"

extern "C" {
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
}
