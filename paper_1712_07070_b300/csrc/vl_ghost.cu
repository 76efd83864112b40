// vl_ghost.cu -- the VL scheme (GAMER-2 section 2.2) on refined levels: the
// predictor's half step on the coarse-fine ghost patches.
//
// The corrector of a group next to a coarse-fine interface reconstructs the
// half-step state U* two cells deep into its ghost patches.  The level's own
// patches get U* from the predictor launch of the step kernel; the ghost
// cells get it here, from the interpolated U^n (three cells deep) with the
// same first-order fluxes of cell averages:
//   U*_i = U^n_i - dt/(2 dh) sum_d (F(U_i, U_{i+d}) - F(U_{i-d}, U_i)).
// One CTA per ghost patch; the cells are the two layers its groups read
// along each outer direction (the ghost box of depth 4 shrunk to depth 2).
#include <cuda_runtime.h>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

namespace amrh {
namespace {

struct VlGhostArgs {
    const double *U;        // the level's U^n
    const double *ghost;    // its interpolated ghost patches
    double *ustar;          // U* of the ghost patches
    const int32_t *info;    // ghost jobs (GHOST_INFO ints; the box at [4])
    const int32_t *gnbr;    // 27 positions around each ghost patch
    int n_ghost;
    double dt;                          // >= 0, or the device CFL dt from smax_in
    const unsigned long long *smax_in;
    double cfl, dh, gamma;
    int limiter, riemann;
    double theta;
    int fallback;
};

constexpr int VG_NT = 128;

template <typename real, int MODE>
__global__ void __launch_bounds__(VG_NT) k_vl_ghost_pred(VlGhostArgs A) {
    __shared__ int nb[27];
    __shared__ double sdt;
    const int tid = threadIdx.x;
    Gas<real> g;
    g.gamma = (real)A.gamma;
    g.gm1 = (real)(A.gamma - 1.0);
    g.inv_gm1 = (real)(1.0 / (A.gamma - 1.0));
    if constexpr (MODE != 0) {
        g.lim = A.limiter;
        g.htheta = (real)(0.5 * A.theta);
    }
    if constexpr (MODE == 1) g.rs = A.riemann == RS_HLLE ? RS_HLLE : (A.riemann == RS_ROE ? RS_ROE : RS_HLLC);
    g.fb = A.fallback;
    if constexpr (MODE == 2) g.rs = RS_EXACT;
    if (tid == 0) {
        double dt = A.dt;
        if (dt < 0.0) dt = A.cfl * A.dh / __longlong_as_double((long long)*A.smax_in);
        sdt = dt;
    }
    __syncthreads();
    const double dtdh = 0.5 * sdt / A.dh;
    const real dtdh_r = (real)dtdh;
    for (int j = blockIdx.x; j < A.n_ghost; j += gridDim.x) {
        __syncthreads();  // the previous patch's reads of nb are done
        if (tid < 27) nb[tid] = A.gnbr[(int64_t)j * 27 + tid];
        __syncthreads();
        const double *own = A.ghost + (int64_t)j * PSLOT;
        // conserved state of cell (x, y, z) of this patch's 3x3x3 neighbourhood
        // (each coordinate -8..15); a position with no data gives `fallback`
        auto cell = [&](int x, int y, int z, const real *fallback, real u[NV]) {
            const double *src = own;
            if ((unsigned)x > 7u || (unsigned)y > 7u || (unsigned)z > 7u) {
                const int s = nb[((x + 8) >> 3) + 3 * ((y + 8) >> 3) + 9 * ((z + 8) >> 3)];
                src = s >= 0 ? A.U + (int64_t)s * PSLOT : (s <= -2 ? A.ghost + (int64_t)(-2 - s) * PSLOT : nullptr);
            }
            if (!src) {
#pragma unroll
                for (int v = 0; v < NV; v++) u[v] = fallback[v];
                return;
            }
            const int off = ((z + 8) & 7) * 64 + ((y + 8) & 7) * 8 + ((x + 8) & 7);
#pragma unroll
            for (int v = 0; v < NV; v++) u[v] = to_real<real>(src[v * PV + off]);
        };
        const int box = A.info[(int64_t)GHOST_INFO * j + 4];
        int lo[3], n[3];
        for (int d = 0; d < 3; d++) {
            const int l = (box >> (4 * d)) & 15, h = (box >> (12 + 4 * d)) & 15;
            lo[d] = l == 4 ? 6 : l;
            n[d] = (h == 4 ? 2 : h) - lo[d];
        }
        const int total = n[0] * n[1] * n[2];
        for (int i = tid; i < total; i += VG_NT) {
            const int x = lo[0] + i % n[0], y = lo[1] + (i / n[0]) % n[1], z = lo[2] + i / (n[0] * n[1]);
            const int off = z * 64 + y * 8 + x;
            real ui[NV], um[NV], up[NV], fm[NV], fp[NV], tot[NV];
            cell(x, y, z, ui, ui);
            // ((F_x+ - F_x-) + (F_y+ - F_y-) - F_z-) + F_z+, the step kernel's order
            cell(x - 1, y, z, ui, um);
            cell(x + 1, y, z, ui, up);
            face_flux<0>(um, ui, fm, g);
            face_flux<0>(ui, up, fp, g);
#pragma unroll
            for (int v = 0; v < NV; v++) tot[v] = fp[v] - fm[v];
            cell(x, y - 1, z, ui, um);
            cell(x, y + 1, z, ui, up);
            face_flux<1>(um, ui, fm, g);
            face_flux<1>(ui, up, fp, g);
#pragma unroll
            for (int v = 0; v < NV; v++) tot[v] = tot[v] + (fp[v] - fm[v]);
            cell(x, y, z - 1, ui, um);
            cell(x, y, z + 1, ui, up);
            face_flux<2>(um, ui, fm, g);
            face_flux<2>(ui, up, fp, g);
            double *o = A.ustar + (int64_t)j * PSLOT;
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const real t = (tot[v] - fm[v]) + fp[v];
                const double uo = own[v * PV + off];
                if constexpr (sizeof(real) == sizeof(double)) o[v * PV + off] = uo - dtdh * t;
                else o[v * PV + off] = uo - f2d_bits(dtdh_r * t);
            }
        }
    }
}

template <typename real>
void launch_vg(int mode, const VlGhostArgs &A, int grid, cudaStream_t s) {
    if (mode == 0) k_vl_ghost_pred<real, 0><<<grid, VG_NT, 0, s>>>(A);
    else if (mode == 1) k_vl_ghost_pred<real, 1><<<grid, VG_NT, 0, s>>>(A);
    else k_vl_ghost_pred<real, 2><<<grid, VG_NT, 0, s>>>(A);
}

}  // namespace

amr_status launch_vl_ghost_pred(amr_hydro_ctx *c, int level, const StepParams &P) {
    Level &L = c->lv[level];
    if (!L.n_ghost) return AMR_OK;
    if (!L.ghost_ustar.p || !L.ghost_nbr.p) return AMR_E_INVAL;
    VlGhostArgs A;
    A.U = P.U_old;
    A.ghost = L.ghost.p;
    A.ustar = L.ghost_ustar.p;
    A.info = L.ghost_info.p;
    A.gnbr = L.ghost_nbr.p;
    A.n_ghost = L.n_ghost;
    A.dt = P.dt;
    A.smax_in = P.smax_in;
    A.cfl = P.cfl;
    A.dh = P.dh;
    A.gamma = P.gamma;
    A.limiter = P.limiter;
    A.riemann = P.riemann;
    A.theta = P.theta;
    A.fallback = P.fallback;
    const int grid = L.n_ghost < 8 * c->n_sm ? L.n_ghost : 8 * c->n_sm;
    const int mode = scheme_mode(P.limiter, P.riemann);
    if (c->prm.prec == AMR_FP64) launch_vg<double>(mode, A, grid, c->stream);
    else launch_vg<float>(mode, A, grid, c->stream);
    return cuda_fail(cudaGetLastError(), "k_vl_ghost_pred");
}

}  // namespace amrh
