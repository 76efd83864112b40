// fallback.cu -- remedies (ii) and (iii) of GAMER-2 section 2.2 for cells the
// step left unphysical (rho <= 0 or P <= 0).  The step kernel appends such a
// cell to a device list instead of counting it; this kernel, launched after
// the step on the same stream, recomputes each listed cell from U^n:
//   (ii)  first order in space and time, unsplit:
//         U^n - (dt/dh) sum_d [F_d(U_i, U_i+1) - F_d(U_i-1, U_i)] with the
//         selected Riemann solver on cell averages;
//   (iii) if that is unphysical too, first order dimensionally split: an x
//         sweep of U^n over the cell's 3x3x3 neighbourhood, a y sweep of that
//         result, a z sweep of that;
// in FP64 in both precision modes, and counts the cells still unphysical
// (remedy iv, the level retry, is the host's).  The neighbourhood is read
// through the level's neighbour table (corner positions included when the
// remedies are on).  Keeping this out of the step kernel leaves its
// register allocation untouched.
#include <cuda_runtime.h>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

namespace amrh {

namespace {

__device__ __forceinline__ bool physical(const double u[NV]) {
    return pos_finite(u[0]) && pos_finite(2.0 * u[0] * u[4] - (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]));
}

// First-order update along D of the middle of three cells.
template <int D>
__device__ __forceinline__ void fo_sweep(const double vm[NV], const double v0[NV], const double vp[NV], double r,
                                         const Gas<double> &g, double out[NV]) {
    double fp[NV], fm[NV];
    face_flux<D>(v0, vp, fp, g);
    face_flux<D>(vm, v0, fm, g);
#pragma unroll
    for (int v = 0; v < NV; v++) out[v] = v0[v] - r * (fp[v] - fm[v]);
}

__global__ void k_cell_remedies(const double *__restrict__ U0, double *__restrict__ U_new,
                                const int32_t *__restrict__ nbr, const double *__restrict__ ghost,
                                const int64_t *__restrict__ list, const unsigned long long *count, int64_t cap,
                                double dt_in, double cfl, const unsigned long long *smax_in, double dh,
                                double gamma, int rs, int roe_check, int cfl1, unsigned long long *smax_out,
                                unsigned long long *n_bad) {
    Gas<double> g;
    g.gamma = gamma;
    g.gm1 = gamma - 1.0;
    g.inv_gm1 = 1.0 / (gamma - 1.0);
    g.rs = rs;
    g.fb = roe_check;
    const int64_t n = min((int64_t)*count, cap);
    // the step's dt: the host's, or the device's CFL dt as the step computed it
    const double dt = dt_in >= 0.0 ? dt_in : cfl * dh / __longlong_as_double((long long)*smax_in);
    const double r = dt / dh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = list[i];
        const int64_t slot = base / PSLOT;
        const int off = (int)(base % PSLOT), p = (int)(slot & 7);
        const int64_t grp = slot >> 3;
        // the cell's coordinates in its group's 16^3 tile
        const int x = (p & 1) * PS + (off & 7), y = ((p >> 1) & 1) * PS + ((off >> 3) & 7),
                  z = (p >> 2) * PS + (off >> 6);
        double B[3][3][3][NV];  // U^n at tile cells (x+i-1, y+j-1, z+k-1): B[k][j][i]
        for (int k = 0; k < 3; k++)
            for (int j = 0; j < 3; j++)
                for (int a = 0; a < 3; a++) {
                    const int tx = x + a - 1, ty = y + j - 1, tz = z + k - 1;
                    const int q = ((tx + PS) >> 3) + 4 * ((ty + PS) >> 3) + 16 * ((tz + PS) >> 3);
                    const int s = nbr[grp * 64 + q];
                    const double *src = s >= 0 ? U0 + (int64_t)s * PSLOT
                                               : (s <= -2 ? ghost + (int64_t)(-2 - s) * PSLOT : nullptr);
                    const int o = ((tz + PS) & 7) * 64 + ((ty + PS) & 7) * 8 + ((tx + PS) & 7);
#pragma unroll
                    for (int v = 0; v < NV; v++) B[k][j][a][v] = src ? src[v * PV + o] : B[1][1][1][v];
                }
        // (ii)
        double out[NV], fp[NV], fm[NV], div[NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
        face_flux<0>(B[1][1][1], B[1][1][2], fp, g);
        face_flux<0>(B[1][1][0], B[1][1][1], fm, g);
#pragma unroll
        for (int v = 0; v < NV; v++) div[v] += fp[v] - fm[v];
        face_flux<1>(B[1][1][1], B[1][2][1], fp, g);
        face_flux<1>(B[1][0][1], B[1][1][1], fm, g);
#pragma unroll
        for (int v = 0; v < NV; v++) div[v] += fp[v] - fm[v];
        face_flux<2>(B[1][1][1], B[2][1][1], fp, g);
        face_flux<2>(B[0][1][1], B[1][1][1], fm, g);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            div[v] += fp[v] - fm[v];
            out[v] = B[1][1][1][v] - r * div[v];
        }
        if (!physical(out)) {  // (iii)
            double X[3][3][NV], Y[3][NV];
            for (int k = 0; k < 3; k++)
                for (int j = 0; j < 3; j++) fo_sweep<0>(B[k][j][0], B[k][j][1], B[k][j][2], r, g, X[k][j]);
            for (int k = 0; k < 3; k++) fo_sweep<1>(X[k][0], X[k][1], X[k][2], r, g, Y[k]);
            fo_sweep<2>(Y[0], Y[1], Y[2], r, g, out);
        }
#pragma unroll
        for (int v = 0; v < NV; v++) U_new[base + v * PV] = out[v];
        if (physical(out)) {
            bool ok;
            const double sp = cfl_speed(out, g, ok, cfl1 != 0);
            atomicMax(smax_out, (unsigned long long)__double_as_longlong(sp));
        } else {
            atomicAdd(n_bad, 1ull);
        }
    }
}

}  // namespace

// Remedies (ii)-(iii) for the cells the step launch P listed, then an empty
// list for the next launch.  Base: the U^n slots the step read (U_base for
// the VL corrector).
amr_status launch_cell_remedies(amr_hydro_ctx *c, const StepParams &P, const double *base, int cfl1,
                                cudaStream_t s) {
    if (!P.fb_list) return AMR_OK;
    k_cell_remedies<<<c->n_sm * 2, 128, 0, s>>>(base, P.U_new, P.nbr, P.ghost, P.fb_list, P.fb_count, P.fb_cap,
                                                  P.dt, P.cfl, P.smax_in, P.dh, P.gamma, P.riemann, P.fallback,
                                                  cfl1, P.smax_out, P.n_bad);
    amr_status st = cuda_fail(cudaGetLastError(), "k_cell_remedies");
    if (st) return st;
    return cuda_fail(cudaMemsetAsync(P.fb_count, 0, sizeof(unsigned long long), s), "memset");
}

}  // namespace amrh
