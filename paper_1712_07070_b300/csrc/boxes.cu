// boxes.cu -- many independent periodic boxes advanced together (the paper's
// section 4.2 runs one periodic Kelvin-Helmholtz domain per node; here many
// such domains of uneven sizes share one GPU).
//
// All groups of all listed boxes form one work list that a single persistent
// launch walks per step; each box takes its own dt of Eq. (CFL2), computed on
// the device from the signal speed its previous step reduced, so a batch of
// steps needs no host synchronisation and is captured once into a CUDA graph
// and replayed.  An autotuner times the launch shapes on the workload (with
// dt = 0, which leaves the state unchanged) and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

using namespace amrh;

namespace {

// Kernel instances: key K = MODE + 3 STAGE, as for the level step kernel.
// the box batch runs the stages up to dual energy (no gravity)
using BoxKeys = std::make_integer_sequence<int, 3 * (ST_MH_DE + 1)>;

template <typename real, int K>
amr_status set_box_smem() {
    return cuda_fail(cudaFuncSetAttribute(k_hydro_step_boxes<real, K % 3, K / 3>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(StageSmem<real, K / 3>)),
                     "box kernel smem attribute");
}
template <typename real, int... K>
amr_status set_box_smem_all(std::integer_sequence<int, K...>) {
    amr_status st = AMR_OK;
    ((st = st ? st : set_box_smem<real, K>()), ...);
    return st;
}

amr_status configure_box_kernels() {
    static DeviceOnce once;
    return once_per_device(once, [] {
        amr_status st;
        if ((st = set_box_smem_all<double>(BoxKeys{})) || (st = set_box_smem_all<float>(BoxKeys{}))) return st;
        return AMR_OK;
    });
}

template <typename real, int K>
int box_occupancy_k() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hydro_step_boxes<real, K % 3, K / 3>, StepCfg<real>::NT,
                                                  sizeof(StageSmem<real, K / 3>));
    return n;
}
template <typename real, int... K>
int box_occupancy(int lo, int hi, std::integer_sequence<int, K...>) {
    int n = 1 << 20;
    ((n = (K / 3 >= lo && K / 3 <= hi) ? std::min(n, box_occupancy_k<real, K>()) : n), ...);
    return n > 0 ? n : 1;
}

// Resident CTAs per SM of the instances the context's scheme launches.
int resident_per_sm(int prec, int scheme, int recon, int dual_energy) {
    int lo, hi;
    scheme_stages(scheme, recon, dual_energy, lo, hi);
    return prec == AMR_FP64 ? box_occupancy<double>(lo, hi, BoxKeys{}) : box_occupancy<float>(lo, hi, BoxKeys{});
}

template <typename real, int K>
void launch_boxes_one(const BoxLaunch &B, int grid, cudaStream_t s) {
    k_hydro_step_boxes<real, K % 3, K / 3><<<grid, StepCfg<real>::NT, sizeof(StageSmem<real, K / 3>), s>>>(B);
}
template <typename real, int... K>
void launch_boxes_key(int key, const BoxLaunch &B, int grid, cudaStream_t s, std::integer_sequence<int, K...>) {
    ((key == K ? launch_boxes_one<real, K>(B, grid, s) : void()), ...);
}

// One step of the batch: one launch (MUSCL-Hancock, CTU) or the VL predictor
// and corrector launches.
amr_status launch_boxes(amr_hydro_ctx *c, const BoxLaunch &B, int grid, cudaStream_t s) {
    const int mode = scheme_mode(B.limiter, B.riemann);
    int lo, hi;
    scheme_stages(c->prm.scheme, c->prm.recon, c->prm.dual_energy, lo, hi);
    for (int stage = lo; stage <= hi; stage++) {
        if (c->prm.prec == AMR_FP64)
            launch_boxes_key<double>(mode + 3 * stage, B, grid, s, BoxKeys{});
        else
            launch_boxes_key<float>(mode + 3 * stage, B, grid, s, BoxKeys{});
        amr_status st = cuda_fail(cudaGetLastError(), "k_hydro_step_boxes");
        if (st) return st;
    }
    return AMR_OK;
}

__global__ void k_zero_box_out(BoxDesc *desc, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int r = (desc[i].ring0 + 1) % 3;
        desc[i].scal[r] = 0ull;
        desc[i].scal[3 + r] = 0ull;
    }
}

// (box, group) work list: box-major or interleaved round-robin over boxes.
std::vector<int32_t> make_work(amr_hydro_ctx *c, const std::vector<int> &ids, int interleave) {
    std::vector<int32_t> w;
    if (!interleave) {
        for (size_t i = 0; i < ids.size(); i++)
            for (int g = 0; g < c->boxes[ids[i]].n_groups; g++) w.insert(w.end(), {(int32_t)i, g});
    } else {
        int gmax = 0;
        for (int id : ids) gmax = std::max(gmax, c->boxes[id].n_groups);
        for (int g = 0; g < gmax; g++)
            for (size_t i = 0; i < ids.size(); i++)
                if (g < c->boxes[ids[i]].n_groups) w.insert(w.end(), {(int32_t)i, g});
    }
    return w;
}

amr_status upload_work(amr_hydro_ctx *c, const std::vector<int> &ids, int interleave) {
    std::vector<int> key(ids);
    key.push_back(interleave);
    if (key == c->plan_key) return AMR_OK;
    std::vector<int32_t> w = make_work(c, ids, interleave);
    amr_status st = c->box_plan.reserve(w.size());
    if (st) return st;
    if ((st = cuda_fail(cudaMemcpy(c->box_plan.p, w.data(), 4 * w.size(), cudaMemcpyHostToDevice), "h2d work")))
        return st;
    c->plan_key = key;
    return AMR_OK;
}

}  // namespace

extern "C" {

amr_status amr_hydro_set_box(amr_hydro_ctx *c, int box_id, int n, double *U_a, double *U_b) {
    if (!c || box_id < 0 || box_id >= MAX_BOXES || n <= 0 || n % 16 || !U_a || !U_b || U_a == U_b)
        return AMR_E_INVAL;
    Box &B = c->boxes[box_id];
    const int np[3] = {n / 8, n / 8, n / 8};
    const int64_t npatch = (int64_t)np[0] * np[1] * np[2];
    std::vector<int32_t> corner(3 * npatch), sib(26 * npatch), nbr;
    std::vector<GhostInfo> ghosts;
    amr_status st = build_uniform_tables(np, corner.data(), sib.data(), nullptr, nullptr);
    if (st) return st;
    const int cells[3] = {n, n, n};
    if ((st = build_nbr_plan(0, (int)npatch, corner.data(), sib.data(), nullptr, cells, nbr, ghosts))) return st;
    if ((st = B.nbr.reserve(nbr.size()))) return st;
    if (c->prm.scheme == AMR_SCHEME_VL && (st = B.ustar.reserve((size_t)npatch * PSLOT))) return st;
    if ((st = cuda_fail(cudaMemcpy(B.nbr.p, nbr.data(), 4 * nbr.size(), cudaMemcpyHostToDevice), "h2d"))) return st;
    if ((st = cuda_fail(cudaMemset(c->scal.p + SCAL_BOX0 + SCAL_PER * box_id, 0, 8 * SCAL_PER), "memset"))) return st;
    B.n = n;
    B.n_groups = (int)(npatch / 8);
    B.U[0] = U_a;
    B.U[1] = U_b;
    B.S[0] = B.S[1] = nullptr;  // dual energy: amr_hydro_set_box_entropy
    B.cur = 0;
    B.ring = 0;
    B.speed_valid = false;
    c->plan_key.clear();
    c->tune_key.clear();
    c->graph_key.clear();
    return AMR_OK;
}

amr_status amr_hydro_set_box_entropy(amr_hydro_ctx *c, int box_id, double *S_a, double *S_b) {
    if (!c || box_id < 0 || box_id >= MAX_BOXES || !c->prm.dual_energy) return AMR_E_INVAL;
    Box &B = c->boxes[box_id];
    if (!B.n || !S_a || !S_b || S_a == S_b) return AMR_E_INVAL;
    B.S[B.cur] = S_a;
    B.S[1 - B.cur] = S_b;
    B.speed_valid = false;
    c->graph_key.clear();
    return AMR_OK;
}

amr_status amr_hydro_box_state(amr_hydro_ctx *c, int box_id, int *cur) {
    if (!c || !cur || box_id < 0 || box_id >= MAX_BOXES || !c->boxes[box_id].n) return AMR_E_INVAL;
    *cur = c->boxes[box_id].cur;
    return AMR_OK;
}

amr_status amr_hydro_box_tuning(amr_hydro_ctx *c, int *grid, int *chunked, int *interleave, float *ms_per_step) {
    if (!c) return AMR_E_INVAL;
    if (grid) *grid = c->tune.grid;
    if (chunked) *chunked = c->tune.chunked;
    if (interleave) *interleave = c->tune.interleave;
    if (ms_per_step) *ms_per_step = c->tune.ms;
    return AMR_OK;
}

amr_status amr_hydro_advance_boxes(amr_hydro_ctx *c, int n_boxes, const int *box_ids, int n_steps,
                                   double *dt_log) {
    if (!c || n_boxes <= 0 || n_boxes > MAX_BOXES || !box_ids || n_steps < 0) return AMR_E_INVAL;
    std::vector<int> ids(box_ids, box_ids + n_boxes);
    {
        std::vector<int> sorted(ids);
        std::sort(sorted.begin(), sorted.end());
        for (int i = 0; i < n_boxes; i++) {
            if (sorted[i] < 0 || sorted[i] >= MAX_BOXES || !c->boxes[sorted[i]].n) return AMR_E_INVAL;
            if (i && sorted[i] == sorted[i - 1]) return AMR_E_INVAL;
            if (c->prm.dual_energy && !c->boxes[sorted[i]].S[0]) return AMR_E_INVAL;  // no entropy fields
        }
    }
    if (!n_steps) return AMR_OK;
    amr_status st = configure_box_kernels();
    if (st) return st;
    cudaStream_t s = c->stream;
    // initial signal speeds of boxes whose state is new
    for (int id : ids) {
        Box &B = c->boxes[id];
        if (B.speed_valid) continue;
        unsigned long long *sc = c->scal.p + SCAL_BOX0 + SCAL_PER * id;
        if ((st = cuda_fail(cudaMemsetAsync(sc, 0, 8 * SCAL_PER, s), "memset"))) return st;
        if ((st = launch_max_speed(c->prm.prec, B.U[B.cur], (int64_t)B.n_groups * 8, c->prm.gamma,
                                   c->prm.scheme == AMR_SCHEME_CTU, sc + B.ring,
                                   sc + 3 + B.ring, c->n_sm, s)))
            return st;
        B.speed_valid = true;
    }
    // descriptors (read by the kernels at run time: the graph stays valid)
    std::vector<BoxDesc> desc(n_boxes);
    int64_t total_groups = 0;
    for (int i = 0; i < n_boxes; i++) {
        Box &B = c->boxes[ids[i]];
        desc[i].U[0] = B.U[0];
        desc[i].U[1] = B.U[1];
        desc[i].S[0] = B.S[0];
        desc[i].S[1] = B.S[1];
        desc[i].ustar = B.ustar.p;
        desc[i].nbr = B.nbr.p;
        desc[i].scal = c->scal.p + SCAL_BOX0 + SCAL_PER * ids[i];
        desc[i].dh = 1.0 / B.n;
        desc[i].n_groups = B.n_groups;
        desc[i].cur0 = B.cur;
        desc[i].ring0 = B.ring;
        desc[i].log_index = i;
        total_groups += B.n_groups;
    }
    if ((st = c->box_desc.reserve(sizeof(BoxDesc) * n_boxes))) return st;
    if ((st = cuda_fail(cudaMemcpyAsync(c->box_desc.p, desc.data(), sizeof(BoxDesc) * n_boxes, cudaMemcpyHostToDevice, s),
                        "h2d desc")))
        return st;
    BoxLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.desc = (const BoxDesc *)c->box_desc.p;
    L.cfl = c->prm.cfl;
    L.gamma = c->prm.gamma;
    L.limiter = c->prm.limiter;
    L.riemann = c->prm.riemann;
    L.theta = c->prm.minmod_coeff;
    L.fallback = c->prm.fallback;
    L.n_boxes = n_boxes;
    L.de_xi = c->prm.dual_xi;

    // autotune the launch shape once per box set
    if (c->tune_key != ids) {
        const char *env = std::getenv("AMR_HYDRO_AUTOTUNE");
        const bool tune = !(env && env[0] == '0');
        const int res = resident_per_sm(c->prm.prec, c->prm.scheme, c->prm.recon, c->prm.dual_energy);
        std::vector<BoxTune> cands;
        for (int mult : {1, res, 2 * res, 4 * res})
            for (int chunked : {0, 1})
                for (int inter : {0, 1}) {
                    BoxTune t;
                    t.grid = c->n_sm * mult;
                    t.chunked = chunked;
                    t.interleave = inter;
                    if (t.grid > total_groups) t.grid = (int)total_groups;
                    cands.push_back(t);
                }
        if (!tune) cands.assign(1, cands[2]);  // resident grid, grid-stride, box-major
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        BoxTune best;
        best.ms = 1e30f;
        for (BoxTune &t : cands) {
            if ((st = upload_work(c, ids, t.interleave))) break;
            BoxLaunch T = L;
            T.work = (const int2 *)c->box_plan.p;
            T.n_work = (int)total_groups;
            T.chunked = t.chunked;
            T.dt_override = 0.0;  // U_new = U_old: the state is untouched
            T.step = 0;
            if (tune) {
                if ((st = launch_boxes(c, T, t.grid, s))) break;
                cudaEventRecord(e0, s);
                for (int k = 0; k < 2; k++)
                    if ((st = launch_boxes(c, T, t.grid, s))) break;
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&t.ms, e0, e1);
                t.ms *= 0.5f;
            }
            if (t.ms < best.ms) best = t;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st) return st;
        c->tune = best;
        c->tune_key = ids;
        c->graph_key.clear();
    }
    if ((st = upload_work(c, ids, c->tune.interleave))) return st;
    L.work = (const int2 *)c->box_plan.p;
    L.n_work = (int)total_groups;
    L.chunked = c->tune.chunked;
    L.dt_override = -1.0;
    L.dt_log = dt_log;

    // capture n_steps launches into a graph once; replay it afterwards
    std::vector<long long> gkey(ids.begin(), ids.end());
    gkey.push_back(n_steps);
    gkey.push_back((long long)(intptr_t)dt_log);
    gkey.push_back(c->tune.grid);
    gkey.push_back(c->tune.chunked);
    gkey.push_back(c->tune.interleave);
    // the first step's reduction slots start at zero (after any tuning launch)
    k_zero_box_out<<<(n_boxes + 127) / 128, 128, 0, s>>>((BoxDesc *)c->box_desc.p, n_boxes);
    if ((st = cuda_fail(cudaGetLastError(), "k_zero_box_out"))) return st;
    if (gkey != c->graph_key || !c->graph_exec) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        if (!c->capture_stream &&
            (st = cuda_fail(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "stream")))
            return st;
        // the capture stream waits for nothing; the graph runs on c->stream
        if ((st = cuda_fail(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal), "capture")))
            return st;
        amr_status cap = AMR_OK;
        for (int k = 0; k < n_steps && !cap; k++) {
            BoxLaunch S = L;
            S.step = k;
            cap = launch_boxes(c, S, c->tune.grid, c->capture_stream);
        }
        cudaGraph_t graph = nullptr;
        st = cuda_fail(cudaStreamEndCapture(c->capture_stream, &graph), "end capture");
        if (cap) {
            if (graph) cudaGraphDestroy(graph);
            return cap;
        }
        if (st) return st;
        st = cuda_fail(cudaGraphInstantiate(&c->graph_exec, graph, 0), "instantiate");
        cudaGraphDestroy(graph);
        if (st) return st;
        c->graph_key = gkey;
    }
    if ((st = cuda_fail(cudaGraphLaunch(c->graph_exec, s), "graph launch"))) return st;
    for (int id : ids) {
        Box &B = c->boxes[id];
        B.cur = (B.cur + n_steps) & 1;
        B.ring = (B.ring + n_steps) % 3;
    }
    return AMR_OK;
}

}  // extern "C"
