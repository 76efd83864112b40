// amr_hydro.cu -- C ABI of the B300-native GAMER-2 patch-group hydro update:
// context, per-level neighbour plans, launches.  The ABI is declared and
// documented in include/amr_hydro.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

using namespace amrh;

namespace amrh {

const char *status_str(amr_status s) {
    switch (s) {
        case AMR_OK: return "ok";
        case AMR_E_INVAL: return "invalid argument";
        case AMR_E_NOMEM: return "out of memory";
        case AMR_E_CUDA: return "CUDA error";
        case AMR_E_UNPHYSICAL: return "unphysical state (rho<=0 or P<=0)";
        case AMR_E_TIMEOUT: return "bounded device wait timed out";
        case AMR_E_NESTING: return "proper-nesting violation";
    }
    return "unknown status";
}

amr_status cuda_fail(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return AMR_OK;
    std::fprintf(stderr, "amr_hydro: %s: %s\n", where, cudaGetErrorString(e));
    return AMR_E_CUDA;
}

template <typename T>
amr_status DevBuf<T>::reserve(size_t n) {
    if (n <= cap) return AMR_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, sizeof(T) * n) != cudaSuccess) {
        cudaGetLastError();
        return AMR_E_NOMEM;
    }
    cap = n;
    return AMR_OK;
}
template <typename T>
void DevBuf<T>::release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}
template struct DevBuf<int32_t>;
template struct DevBuf<int64_t>;
template struct DevBuf<double>;
template struct DevBuf<unsigned long long>;
template struct DevBuf<uint8_t>;
template struct DevBuf<uint32_t>;

size_t step_smem_bytes(int prec) {
    return prec == AMR_FP64 ? sizeof(StepSmem<double>) : sizeof(StepSmem<float>);
}

// Kernel instances: key K = MODE + 3 STAGE (scheme_mode of the limiter and
// solver; the stages ST_MH .. ST_CTU_PPM).
using StepKeys = std::make_integer_sequence<int, 3 * N_STAGES>;

template <typename real, int K>
static amr_status set_step_smem() {
    return cuda_fail(cudaFuncSetAttribute(k_hydro_step<real, K % 3, K / 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(StageSmem<real, K / 3>)),
                     "step kernel smem attribute");
}
template <typename real, int... K>
static amr_status set_step_smem_all(std::integer_sequence<int, K...>) {
    amr_status st = AMR_OK;
    ((st = st ? st : set_step_smem<real, K>()), ...);
    return st;
}

amr_status configure_kernels() {
    static DeviceOnce once;
    return once_per_device(once, [] {
        amr_status st;
        if ((st = set_step_smem_all<double>(StepKeys{})) || (st = set_step_smem_all<float>(StepKeys{}))) return st;
        return AMR_OK;
    });
}

template <typename real, int K>
static int step_occupancy_k() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hydro_step<real, K % 3, K / 3>, StepCfg<real>::NT,
                                                  sizeof(StageSmem<real, K / 3>));
    return n;
}
template <typename real, int... K>
static int step_occupancy(int stage_lo, int stage_hi, std::integer_sequence<int, K...>) {
    int n = 1 << 20;
    ((n = (K / 3 >= stage_lo && K / 3 <= stage_hi) ? std::min(n, step_occupancy_k<real, K>()) : n), ...);
    return n > 0 ? n : 1;
}

// The march stages a scheme launches, lo .. hi: MUSCL-Hancock or CTU (PLM or
// PPM), or the two VL launches.
void scheme_stages(int scheme, int recon, int dual_energy, int &lo, int &hi) {
    const bool ppm = recon == AMR_RECON_PPM;
    if (dual_energy) {
        lo = hi = ST_MH_DE;
    } else if (scheme == AMR_SCHEME_VL) {
        lo = ST_VL_PRED;
        hi = ST_VL_CORR;
    } else if (scheme == AMR_SCHEME_CTU) {
        lo = hi = ppm ? ST_CTU_PPM : ST_CTU;
    } else {
        lo = hi = ppm ? ST_MH_PPM : ST_MH;
    }
}

// Number of resident step CTAs per SM of a scheme's instances, for sizing a
// persistent grid.
int step_blocks_per_sm(int prec, int scheme, int recon, int dual_energy) {
    int lo, hi;
    scheme_stages(scheme, recon, dual_energy, lo, hi);
    return prec == AMR_FP64 ? step_occupancy<double>(lo, hi, StepKeys{}) : step_occupancy<float>(lo, hi, StepKeys{});
}

template <typename real, int K>
static void launch_step_one(const StepParams &P, int grid, cudaStream_t s) {
    k_hydro_step<real, K % 3, K / 3><<<grid, StepCfg<real>::NT, sizeof(StageSmem<real, K / 3>), s>>>(P);
}
template <typename real, int... K>
static void launch_step_key(int key, const StepParams &P, int grid, cudaStream_t s, std::integer_sequence<int, K...>) {
    ((key == K ? launch_step_one<real, K>(P, grid, s) : void()), ...);
}
template <typename real>
static void launch_step_k(const StepParams &P, int grid, cudaStream_t s) {
    launch_step_key<real>(scheme_mode(P.limiter, P.riemann) + 3 * P.stage, P, grid, s, StepKeys{});
}

amr_status launch_step(amr_hydro_ctx *c, const StepParams &P, int grid) {
    if (P.n_work == 0) return AMR_OK;
    if (c->prm.prec == AMR_FP64)
        launch_step_k<double>(P, grid, c->stream);
    else
        launch_step_k<float>(P, grid, c->stream);
    return cuda_fail(cudaGetLastError(), "k_hydro_step launch");
}

// Launch the step kernel on a stream without a context (grid capped at the
// resident-CTA count of the current device).  Allocates nothing.
amr_status launch_step_raw(int prec, const StepParams &P, cudaStream_t stream) {
    amr_status st = configure_kernels();
    if (st) return st;
    if (P.n_work == 0) return AMR_OK;
    int dev = 0, n_sm = 0;
    if ((st = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice"))) return st;
    if ((st = cuda_fail(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "sm count")))
        return st;
    const int cap = n_sm * step_blocks_per_sm(prec, AMR_SCHEME_MH, AMR_RECON_PLM, 0);
    const int grid = P.n_work < cap ? P.n_work : cap;
    if (prec == AMR_FP64)
        launch_step_k<double>(P, grid, stream);
    else
        launch_step_k<float>(P, grid, stream);
    return cuda_fail(cudaGetLastError(), "k_hydro_step launch");
}

}  // namespace amrh

// ---------------------------------------------------------------------------
// reductions and layout kernels

namespace {

template <typename real>
__global__ void k_max_speed(const double *__restrict__ U, int64_t n_slots, double gamma, int cfl1,
                            unsigned long long *smax, unsigned long long *n_bad) {
    Gas<real> g;
    g.gamma = (real)gamma;
    g.gm1 = (real)(gamma - 1.0);
    g.inv_gm1 = (real)(1.0 / (gamma - 1.0));
    double m = 0.0;
    unsigned bad = 0;
    const int64_t ncell = n_slots * PV;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ncell;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / PV, c = i % PV;
        real u[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) u[v] = to_real<real>(U[s * PSLOT + v * PV + c]);
        bool ok;
        const real sp = cfl_speed(u, g, ok, cfl1 != 0);
        if (!ok) bad++;
        else if ((double)sp > m) m = (double)sp;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(smax, (unsigned long long)__double_as_longlong(m));
        if (bad) atomicAdd(n_bad, (unsigned long long)bad);
    }
}

__global__ void k_dt_from_speed(const unsigned long long *smax, const unsigned long long *n_bad,
                                double cfl, double dh, double *dt_out) {
    const double s = __longlong_as_double((long long)*smax);
    *dt_out = (*n_bad || !(s > 0.0)) ? -1.0 : cfl * dh / s;
}

// dense [5][nz][ny][nx] <-> uniform patch layout
__global__ void k_pack(double *__restrict__ dense, int nx, int ny, int nz,
                       double *__restrict__ patches, int to_patches) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int ngx = nx / 16, ngy = ny / 16;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        const int64_t g = (x >> 4) + ngx * ((int64_t)(y >> 4) + (int64_t)ngy * (z >> 4));
        const int64_t slot = 8 * g + ((x >> 3) & 1) + 2 * ((y >> 3) & 1) + 4 * ((z >> 3) & 1);
        const int64_t off = slot * PSLOT + (z & 7) * 64 + (y & 7) * 8 + (x & 7);
        for (int v = 0; v < NV; v++) {
            if (to_patches) patches[off + v * PV] = dense[v * n + i];
            else dense[v * n + i] = patches[off + v * PV];
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI

extern "C" {

const char *amr_hydro_strerror(amr_status s) { return status_str(s); }

amr_status amr_hydro_init(const amr_hydro_params *p, void *stream, amr_hydro_ctx **out) {
    if (!p || !out) return AMR_E_INVAL;
    *out = nullptr;
    if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || p->lmax < 0 || p->lmax > 7) return AMR_E_INVAL;
    if (p->prec != AMR_FP64 && p->prec != AMR_FP32_ACC64) return AMR_E_INVAL;
    if (p->max_patches <= 0 || p->max_patches % 8) return AMR_E_INVAL;
    if (p->limiter < AMR_LIM_VANLEER || p->limiter > AMR_LIM_VL_GMINMOD) return AMR_E_INVAL;
    if (p->riemann < AMR_RS_HLLC || p->riemann > AMR_RS_EXACT) return AMR_E_INVAL;
    if (p->minmod_coeff != 0.0 && !(p->minmod_coeff >= 1.0 && p->minmod_coeff <= 2.0)) return AMR_E_INVAL;
    if (p->scheme < AMR_SCHEME_MH || p->scheme > AMR_SCHEME_CTU) return AMR_E_INVAL;
    if (p->recon != AMR_RECON_PLM && p->recon != AMR_RECON_PPM) return AMR_E_INVAL;
    if (p->scheme == AMR_SCHEME_VL && p->recon != AMR_RECON_PLM) return AMR_E_INVAL;
    if (p->fallback != 0 && p->fallback != 1) return AMR_E_INVAL;
    if (!(p->dt_min >= 0.0)) return AMR_E_INVAL;
    if (p->dual_energy != 0 && p->dual_energy != 1) return AMR_E_INVAL;
    if (!(p->dual_xi >= 0.0)) return AMR_E_INVAL;
    if (p->gravity_bc != AMR_GRAVITY_PERIODIC && p->gravity_bc != AMR_GRAVITY_ISOLATED) return AMR_E_INVAL;
    if (p->dual_energy && (p->scheme != AMR_SCHEME_MH || p->recon != AMR_RECON_PLM || p->fallback))
        return AMR_E_INVAL;
    for (int d = 0; d < 3; d++) {
        if (p->root_n[d] <= 0 || p->root_n[d] % 16) return AMR_E_INVAL;
        if (!p->periodic[d]) return AMR_E_INVAL;
        if (!(p->box[d] > 0.0)) return AMR_E_INVAL;
    }
    // cubic cells
    const double dh0 = p->box[0] / p->root_n[0];
    for (int d = 1; d < 3; d++)
        if (std::fabs(p->box[d] / p->root_n[d] - dh0) > 1e-12 * dh0) return AMR_E_INVAL;
    amr_status st = configure_kernels();
    if (st) return st;
    amr_hydro_ctx *c = new (std::nothrow) amr_hydro_ctx();
    if (!c) return AMR_E_NOMEM;
    c->prm = *p;
    if (c->prm.minmod_coeff == 0.0) c->prm.minmod_coeff = 1.5;
    if (c->prm.dual_xi == 0.0) c->prm.dual_xi = 1e-2;
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    c->step_bps = step_blocks_per_sm(p->prec, p->scheme, p->recon, p->dual_energy);
    if ((st = c->scal.reserve(SCAL_N))) { amr_hydro_destroy(c); return st; }
    if ((st = c->dtbuf.reserve(3 * (MAX_LEVELS + MAX_BOXES)))) { amr_hydro_destroy(c); return st; }
    if (cudaMallocHost(&c->rg.hcnt, 32 * sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&c->rg.htime, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        amr_hydro_destroy(c);
        return AMR_E_NOMEM;
    }
    if (p->fallback) {
        if ((st = c->fb_list.reserve(FB_CAP)) || (st = c->fb_count.reserve(1)) ||
            (st = cuda_fail(cudaMemsetAsync(c->fb_count.p, 0, 8, c->stream), "memset"))) {
            amr_hydro_destroy(c);
            return st;
        }
    }
    if ((st = cuda_fail(cudaMemsetAsync(c->scal.p, 0, sizeof(unsigned long long) * SCAL_N, c->stream),
                        "memset"))) {
        amr_hydro_destroy(c);
        return st;
    }
    *out = c;
    return AMR_OK;
}

amr_status amr_hydro_destroy(amr_hydro_ctx *c) {
    if (!c) return AMR_E_INVAL;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (auto &L : c->lv) L.release();
    for (auto &B : c->boxes) B.release();
    c->box_plan.release();
    c->box_desc.release();
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->scal.release();
    c->dtbuf.release();
    c->flag_summary.release();
    c->pflag.release();
    c->psum.release();
    c->rg.release();
    c->adjbuf.release();
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    for (cudaStream_t x : c->xfer)
        if (x) cudaStreamDestroy(x);
    for (cudaEvent_t e : c->slab_ev) cudaEventDestroy(e);
    c->hstage[0].release();
    c->hstage[1].release();
    c->fb_list.release();
    c->fb_count.release();
    for (const auto &r : c->phase_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->phase_spare) cudaEventDestroy(e);
    release_poisson(c);
    delete c;
    return AMR_OK;
}

amr_status amr_hydro_get_state(amr_hydro_ctx *c, int level, int *cur, double *t_cur, double *t_prev) {
    if (!c || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    const Level &L = c->lv[level];
    if (!L.n_patches) return AMR_E_INVAL;
    amr_status st = level_time(c, level);
    if (st) return st;
    if (cur) *cur = L.cur;
    if (t_cur) *t_cur = L.t;
    if (t_prev) *t_prev = L.t_prev;
    return AMR_OK;
}

amr_status amr_hydro_min_dt(amr_hydro_ctx *c, int level, double *dt_out) {
    if (!c || !dt_out || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    Level &L = c->lv[level];
    if (!L.n_patches) return AMR_E_INVAL;
    amr_status st = level_speed(c, level);
    if (st) return st;
    unsigned long long *sm = c->scal.p + L.scal0 + L.ring, *nb = c->scal.p + L.scal0 + 3 + L.ring;
    cudaPointerAttributes a;
    const bool dev = cudaPointerGetAttributes(&a, dt_out) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    const double dh = level_dh(c, level);
    if (dev) {
        k_dt_from_speed<<<1, 1, 0, c->stream>>>(sm, nb, c->prm.cfl, dh, dt_out);
        return cuda_fail(cudaGetLastError(), "k_dt_from_speed");
    }
    // into pinned host memory (a pageable copy takes a staging detour)
    unsigned long long *h = reinterpret_cast<unsigned long long *>(c->rg.htime + 4);
    if ((st = cuda_fail(cudaMemcpyAsync(&h[0], sm, 8, cudaMemcpyDeviceToHost, c->stream), "d2h")))
        return st;
    if ((st = cuda_fail(cudaMemcpyAsync(&h[1], nb, 8, cudaMemcpyDeviceToHost, c->stream), "d2h")))
        return st;
    if ((st = cuda_fail(cudaStreamSynchronize(c->stream), "sync"))) return st;
    double s;
    std::memcpy(&s, &h[0], 8);
    if (h[1] || !(s > 0.0)) {
        *dt_out = -1.0;
        return AMR_E_UNPHYSICAL;
    }
    *dt_out = c->prm.cfl * dh / s;
    return AMR_OK;
}

amr_status amr_hydro_pack_uniform(const double *dense, int nx, int ny, int nz, double *patches,
                                  void *stream) {
    if (!dense || !patches || nx <= 0 || ny <= 0 || nz <= 0 || nx % 16 || ny % 16 || nz % 16)
        return AMR_E_INVAL;
    k_pack<<<1184, 256, 0, (cudaStream_t)stream>>>(const_cast<double *>(dense), nx, ny, nz, patches, 1);
    return cuda_fail(cudaGetLastError(), "k_pack");
}

amr_status amr_hydro_unpack_uniform(const double *patches, int nx, int ny, int nz, double *dense,
                                    void *stream) {
    if (!dense || !patches || nx <= 0 || ny <= 0 || nz <= 0 || nx % 16 || ny % 16 || nz % 16)
        return AMR_E_INVAL;
    k_pack<<<1184, 256, 0, (cudaStream_t)stream>>>(const_cast<double *>(dense), nx, ny, nz,
                                                    const_cast<double *>(patches), 0);
    return cuda_fail(cudaGetLastError(), "k_unpack");
}

}  // extern "C"

namespace amrh {

// Max signal speed and unphysical count of n_slots patches into (smax, nbad),
// which the caller has zeroed.
amr_status launch_max_speed(int prec, const double *U, int64_t n_slots, double gamma, int cfl1,
                            unsigned long long *smax, unsigned long long *nbad, int n_sm, cudaStream_t stream) {
    if (prec == AMR_FP64)
        k_max_speed<double><<<n_sm * 8, 256, 0, stream>>>(U, n_slots, gamma, cfl1, smax, nbad);
    else
        k_max_speed<float><<<n_sm * 8, 256, 0, stream>>>(U, n_slots, gamma, cfl1, smax, nbad);
    return cuda_fail(cudaGetLastError(), "k_max_speed");
}

double level_dh(const amr_hydro_ctx *c, int level) {
    return c->prm.box[0] / c->prm.root_n[0] / (double)(1 << level);
}

// Max signal speed of the level's newest state into its scalar slots (reuses
// the value fused into the last step when the state has not changed since).
amr_status level_speed(amr_hydro_ctx *c, int level) {
    Level &L = c->lv[level];
    if (L.speed_valid) return AMR_OK;
    unsigned long long *sm = c->scal.p + L.scal0 + L.ring, *nb = c->scal.p + L.scal0 + 3 + L.ring;
    amr_status st = cuda_fail(cudaMemsetAsync(sm, 0, 8, c->stream), "memset");
    if (st) return st;
    if ((st = cuda_fail(cudaMemsetAsync(nb, 0, 8, c->stream), "memset"))) return st;
    const int grid = c->n_sm * 8;
    const int cfl1 = c->prm.scheme == AMR_SCHEME_CTU;
    if (c->prm.prec == AMR_FP64)
        k_max_speed<double><<<grid, 256, 0, c->stream>>>(L.U[L.cur], L.n_patches, c->prm.gamma, cfl1, sm, nb);
    else
        k_max_speed<float><<<grid, 256, 0, c->stream>>>(L.U[L.cur], L.n_patches, c->prm.gamma, cfl1, sm, nb);
    if ((st = cuda_fail(cudaGetLastError(), "k_max_speed"))) return st;
    L.speed_valid = true;
    return AMR_OK;
}

}  // namespace amrh

// ---- phase timing ------------------------------------------------------------------------

namespace amrh {

static cudaEvent_t phase_event(amr_hydro_ctx *c) {
    if (!c->phase_spare.empty()) {
        cudaEvent_t e = c->phase_spare.back();
        c->phase_spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

PhaseScope::PhaseScope(amr_hydro_ctx *ctx, int ph) : c(ctx), phase(ph) {
    if (!c->timing || c->phase_depth++ > 0) return;
    a = phase_event(c);
    if (!a) return;
    on = cudaEventRecord(a, c->stream) == cudaSuccess;
    if (!on) c->phase_spare.push_back(a);
}

PhaseScope::~PhaseScope() {
    if (!c->timing) return;
    c->phase_depth--;
    if (!on) return;
    cudaEvent_t b = phase_event(c);
    if (b && cudaEventRecord(b, c->stream) == cudaSuccess) {
        c->phase_recs.push_back({phase, a, b});
    } else {
        c->phase_spare.push_back(a);
        if (b) c->phase_spare.push_back(b);
    }
}

}  // namespace amrh

extern "C" amr_status amr_hydro_phase_timing(amr_hydro_ctx *c, int on) {
    if (!c) return AMR_E_INVAL;
    c->timing = on != 0;
    return AMR_OK;
}

extern "C" amr_status amr_hydro_phase_times(amr_hydro_ctx *c, double *ms_out, int64_t *calls_out) {
    if (!c || !ms_out) return AMR_E_INVAL;
    amr_status st = cuda_fail(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize(), "sync");
    if (st) return st;
    for (int k = 0; k < AMR_N_PHASES; k++) {
        ms_out[k] = 0.0;
        if (calls_out) calls_out[k] = 0;
    }
    for (const auto &r : c->phase_recs) {
        float ms = 0.f;
        if (r.phase >= 0 && r.phase < AMR_N_PHASES && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ms_out[r.phase] += ms;
            if (calls_out) calls_out[r.phase]++;
        }
        c->phase_spare.push_back(r.a);
        c->phase_spare.push_back(r.b);
    }
    cudaGetLastError();
    c->phase_recs.clear();
    return AMR_OK;
}
