// adjoint.cu -- discrete adjoint of the uniform periodic step.
#include <cuda_runtime.h>

#include "amr_hydro.h"
#include "ctx.h"

extern "C" amr_status amr_hydro_step_adjoint(amr_hydro_ctx *c, int level, double dt, const double *U_n,
                                             const double *lam_np1, double *lam_n) {
    (void)c; (void)level; (void)dt; (void)U_n; (void)lam_np1; (void)lam_n;
    return AMR_E_INVAL;
}
