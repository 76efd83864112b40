// host_stream.cu -- one step of the uniform periodic root grid from a host
// state to a host state, with the PCIe transfers overlapped with the update.
// GAMER-2 (section 3.1) overlaps the transfer of patch batches with the GPU
// solver through CUDA streams; here the batches are z-slabs of patch groups
// (16 cell planes each, contiguous in the group order), the state stays on the
// device between the transfers, and the step of slab k waits only for the
// slabs it reads (k-1, k, k+1, periodic).  With the VL scheme the predictor
// of slab k waits for the uploads of k-1..k+1 and the corrector of slab k for
// the predictors of k-1..k+1; the correctors run in the order 1, ..., ns-1, 0,
// so the first starts after the first four uploads.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

using namespace amrh;

namespace {

// Dense [5][nz][ny][nx] <-> patch slots (order of amr_hydro_uniform_tables)
// for the cells of planes z0 .. z0+15.
__global__ void k_pack_slab(double *__restrict__ dense, int nx, int ny, int nz, int z0,
                            double *__restrict__ patches, int to_patches) {
    const int plane = nx * ny, n = plane * GE;
    const int64_t nall = (int64_t)plane * nz;
    const int ngx = nx / 16, ngy = ny / 16;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = i % nx, y = (i / nx) % ny, z = z0 + i / plane;
        const int64_t g = (x >> 4) + ngx * ((int64_t)(y >> 4) + (int64_t)ngy * (z >> 4));
        const int64_t slot = 8 * g + ((x >> 3) & 1) + 2 * ((y >> 3) & 1) + 4 * ((z >> 3) & 1);
        const int64_t off = slot * PSLOT + (z & 7) * 64 + (y & 7) * 8 + (x & 7);
        const int64_t di = (int64_t)z0 * plane + i;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            if (to_patches) patches[off + v * PV] = dense[v * nall + di];
            else dense[v * nall + di] = patches[off + v * PV];
        }
    }
}

amr_status ensure_xfer(amr_hydro_ctx *c, int n_ev) {
    amr_status st;
    for (cudaStream_t &x : c->xfer)
        if (!x && (st = cuda_fail(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "stream create")))
            return st;
    while ((int)c->slab_ev.size() < n_ev) {
        cudaEvent_t e;
        if ((st = cuda_fail(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create"))) return st;
        c->slab_ev.push_back(e);
    }
    return AMR_OK;
}

}  // namespace

extern "C" amr_status amr_hydro_advance_host(amr_hydro_ctx *c, const double *U_in, double *U_out, double dt,
                                             double *dt_next) {
    if (!c || !U_in || !U_out) return AMR_E_INVAL;
    if (!(dt >= 0.0) && !(dt < 0.0)) return AMR_E_INVAL;  // NaN
    Level &L = c->lv[0];
    if (!L.n_patches || !L.uniform || L.n_ghost) return AMR_E_INVAL;
    if (c->prm.lmax > 0 && c->lv[1].n_patches) return AMR_E_INVAL;  // refined levels: use the W-cycle
    if (c->prm.dual_energy) return AMR_E_INVAL;  // no host copies of the entropy fields
    const int nx = c->prm.root_n[0], ny = c->prm.root_n[1], nz = c->prm.root_n[2];
    if ((int64_t)nx * ny * GE >= (1LL << 31)) return AMR_E_INVAL;
    const int ns = nz / GE, G = (nx / 16) * (ny / 16);  // slabs, groups per slab
    const int64_t ncell = (int64_t)nx * ny * nz, slab_cells = (int64_t)nx * ny * GE;
    amr_status st;
    if ((st = ensure_xfer(c, 2 * ns))) return st;
    for (auto &b : c->hstage)
        if ((st = b.reserve((size_t)(NV * ncell)))) return st;
    cudaStream_t cs = c->stream, up = c->xfer[0], down = c->xfer[1];
    cudaEvent_t *ev_in = c->slab_ev.data(), *ev_out = c->slab_ev.data() + ns;

    // uploads in the order the slab steps need them: ns-1, 0, 1, ..., ns-2.
    // The staging buffers are free: the previous call returned after its last
    // transfer, and nothing else uses them.
    std::vector<int> order(ns);
    for (int j = 0; j < ns; j++) order[j] = (j + ns - 1) % ns;
    for (int j : order) {
        for (int v = 0; v < NV; v++) {
            const int64_t o = v * ncell + j * slab_cells;
            if ((st = cuda_fail(cudaMemcpyAsync(c->hstage[0].p + o, U_in + o, 8 * slab_cells,
                                                cudaMemcpyHostToDevice, up), "h2d slab")))
                return st;
        }
        if ((st = cuda_fail(cudaEventRecord(ev_in[j], up), "event"))) return st;
    }

    double *Uold = L.U[L.cur], *Unew = L.U[1 - L.cur];
    std::vector<char> packed(ns, 0);
    auto pack = [&](int j) -> amr_status {
        if (packed[j]) return AMR_OK;
        packed[j] = 1;
        amr_status s2 = cuda_fail(cudaStreamWaitEvent(cs, ev_in[j], 0), "wait");
        if (s2) return s2;
        k_pack_slab<<<c->n_sm * 4, 256, 0, cs>>>(c->hstage[0].p, nx, ny, nz, j * GE, Uold, 1);
        return cuda_fail(cudaGetLastError(), "k_pack_slab");
    };
    unsigned long long *sc = c->scal.p + L.scal0;
    const int r_in = L.ring, r_out = (L.ring + 1) % 3, r_clr = (L.ring + 2) % 3;
    if (dt < 0.0) {  // the CFL dt of the input state: every slab first
        for (int j : order)
            if ((st = pack(j))) return st;
        L.speed_valid = false;
        if ((st = level_speed(c, 0))) return st;
    }

    StepParams P;
    std::memset(&P, 0, sizeof(P));
    P.U_old = Uold;
    P.U_new = Unew;
    P.nbr = L.nbr.p;
    P.n_work = G;
    P.dt = dt;
    P.smax_in = sc + r_in;
    P.cfl = c->prm.cfl;
    P.dh = level_dh(c, 0);
    P.gamma = c->prm.gamma;
    P.limiter = c->prm.limiter;
    P.riemann = c->prm.riemann;
    P.theta = c->prm.minmod_coeff;
    P.fallback = c->prm.fallback;
    if (c->prm.fallback) {
        P.fb_count = c->fb_count.p;
        P.fb_list = c->fb_list.p;
        P.fb_cap = FB_CAP;
    }
    P.smax_out = sc + r_out;
    P.n_bad = sc + 3 + r_out;
    P.clear2 = sc + r_clr;  // idempotent: every slab launch zeroes the same two slots
    P.cf.coarse_off = L.n_creg ? L.coarse_off.p : nullptr;
    P.cf.coarse_buf = L.creg.p;
    const int cap = c->n_sm * c->step_bps;
    const int grid = G < cap ? G : cap;
    const bool vl = c->prm.scheme == AMR_SCHEME_VL;
    std::vector<char> predicted(ns, 0);
    StepParams H = P;  // the VL predictor: U^n -> U*, no reductions, no time record
    H.stage = ST_VL_PRED;
    H.U_new = L.ustar.p;
    H.smax_out = H.n_bad = H.clear2 = nullptr;
    H.time_rec = nullptr;
    H.cf = CFRegs{nullptr, nullptr, nullptr, nullptr};
    H.fb_count = nullptr;
    H.fb_list = nullptr;
    auto predict = [&](int j) -> amr_status {  // VL half step of slab j
        if (predicted[j]) return AMR_OK;
        predicted[j] = 1;
        amr_status s2;
        if ((s2 = pack((j + ns - 1) % ns)) || (s2 = pack(j)) || (s2 = pack((j + 1) % ns))) return s2;
        H.work0 = j * G;
        return launch_step(c, H, grid);
    };
    {
        int lo, hi;
        scheme_stages(c->prm.scheme, c->prm.recon, 0, lo, hi);
        P.stage = lo;
    }
    if (vl) {
        P.stage = ST_VL_CORR;
        P.U_base = Uold;
        P.U_old = L.ustar.p;
    }
    for (int i = 0; i < ns; i++) {
        const int k = vl ? (i + 1) % ns : i;
        if (vl) {
            if ((st = predict((k + ns - 1) % ns)) || (st = predict(k)) || (st = predict((k + 1) % ns))) return st;
        } else if ((st = pack((k + ns - 1) % ns)) || (st = pack(k)) || (st = pack((k + 1) % ns))) {
            return st;
        }
        P.work0 = k * G;
        P.time_rec = i == 0 ? c->dtbuf.p : nullptr;  // the level's time advances once
        if ((st = launch_step(c, P, grid))) return st;
        if ((st = launch_cell_remedies(c, P, vl ? P.U_base : P.U_old, stage_ctu(P.stage), cs))) return st;
        k_pack_slab<<<c->n_sm * 4, 256, 0, cs>>>(c->hstage[1].p, nx, ny, nz, k * GE, Unew, 0);
        if ((st = cuda_fail(cudaGetLastError(), "k_unpack_slab"))) return st;
        if ((st = cuda_fail(cudaEventRecord(ev_out[k], cs), "event"))) return st;
        if ((st = cuda_fail(cudaStreamWaitEvent(down, ev_out[k], 0), "wait"))) return st;
        for (int v = 0; v < NV; v++) {
            const int64_t o = v * ncell + k * slab_cells;
            if ((st = cuda_fail(cudaMemcpyAsync(U_out + o, c->hstage[1].p + o, 8 * slab_cells,
                                                cudaMemcpyDeviceToHost, down), "d2h slab")))
                return st;
        }
    }
    unsigned long long smax = 0;
    if ((st = cuda_fail(cudaMemcpyAsync(&smax, sc + r_out, 8, cudaMemcpyDeviceToHost, cs), "d2h speed"))) return st;
    if ((st = cuda_fail(cudaStreamSynchronize(cs), "sync"))) return st;
    if ((st = cuda_fail(cudaStreamSynchronize(down), "sync"))) return st;

    L.cur = 1 - L.cur;
    if (dt >= 0.0 && !L.t_pending) {
        L.t_prev = L.t;
        L.t += dt;
    } else {
        L.t_pending = true;
    }
    L.ring = r_out;
    L.speed_valid = true;
    if (dt_next) {
        double s;
        std::memcpy(&s, &smax, 8);
        *dt_next = s > 0.0 ? c->prm.cfl * P.dh / s : -1.0;
    }
    return AMR_OK;
}
