// ctx.h -- library-internal state behind the opaque amr_hydro_ctx.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <initializer_list>
#include <mutex>
#include <vector>

#include "amr_hydro.h"

namespace amrh {

template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;
    amr_status reserve(size_t n);
    void release();
};

constexpr int MAX_LEVELS = 8;
constexpr int MAX_BOXES = 256;
// Scalar slots (unsigned 64-bit) in ctx->scal, 8 per level and 8 per box:
// a ring of three max-signal-speed slots [0..2] and three unphysical-count
// slots [3..5].  The state of ring position r has its speed in slot r and its
// count in slot 3+r; a step reads r, accumulates into (r+1)%3 and zeroes
// (r+2)%3 for the step after it, so no per-step memset is needed.
constexpr int SCAL_PER = 8;
constexpr int SCAL_LEVEL0 = 0;
constexpr int SCAL_BOX0 = SCAL_PER * MAX_LEVELS;
constexpr int SCAL_N = SCAL_BOX0 + SCAL_PER * MAX_BOXES;

// One coarse-fine ghost patch of a level: its 8^3 cells are interpolated from
// the coarse level around the parent patch `cparent` of the group that needs it.
struct GhostInfo {
    int32_t cparent;  // coarse slot of the neighbouring group's parent
    int32_t qx, qy, qz;  // patch position relative to that group (-1..2)
    int32_t box;      // cells any group reads: 4-bit lo/hi per dim (lo_x | lo_y<<4 | lo_z<<8 |
                      // hi_x<<12 | hi_y<<16 | hi_z<<20), even bounds in 0..8
};
constexpr int GHOST_INFO = 8;  // int32 per ghost-patch job on the device
constexpr int PSLOT_DOUBLES = 5 * 512;  // doubles of one patch slot of the conserved variables

struct Level {
    int n_patches = 0, n_groups = 0;
    double *U[2] = {nullptr, nullptr};
    double *S[2] = {nullptr, nullptr};  // dual-energy entropy fields (amr_hydro_set_entropy)
    int cur = 0;
    double t = 0.0, t_prev = 0.0;
    bool t_pending = false;  // t awaits a device-side dt
    const int32_t *d_corner = nullptr, *d_sib = nullptr, *d_parent = nullptr, *d_child = nullptr;
    std::vector<int32_t> corner, sib, parent, child;  // host mirrors
    DevBuf<int32_t> nbr;        // [n_groups][64]
    DevBuf<int32_t> runs, run_off;  // z-runs of groups (step work items), see build_runs
    int n_runs = 0;
    DevBuf<int32_t> chain_up, chain_len;  // the device plan's z-chains (upper neighbour, head lengths)
    // the groups in (z, y, x) order of their positions (single-group work
    // items of a device-regridded level, whose slots stay in place)
    DevBuf<int32_t> work;
    bool has_work = false;
    DevBuf<double> ustar;       // VL half-step state, [n_patches][5][512]
    DevBuf<double> ghost;       // [n_ghost][5][512]
    DevBuf<int32_t> ghost_info; // [n_ghost][GHOST_INFO]
    // VL on refined levels: the half-step state U* of the ghost patches and
    // each ghost patch's 27 neighbouring patch positions (slot >= 0, ghost
    // -2 - id, none -1)
    DevBuf<double> ghost_ustar;
    DevBuf<int32_t> ghost_nbr;
    DevBuf<double> ghost_S;  // dual energy: the entropy of the ghost patches [n_ghost][512]
    // self-gravity in the W-cycle (grav_amr.cu): potential [slot][512] and
    // acceleration [slot][3][512] at the level's newest (index gc) and
    // previous times, and g^n of the coarse-fine ghost patches
    DevBuf<double> phi[2], gacc[2];
    DevBuf<double> ghost_acc;
    int gc = 0;
    unsigned long long structure = 0;  // bumped whenever a regrid changes the level's patches
    int n_ghost = 0;
    // coarse-fine flux registers (section 2.2 fix-up)
    DevBuf<int64_t> fine_off;    // [n_groups*6]: this level's group faces on coarse-fine interfaces
    DevBuf<double> freg;         // their [5][16][16] blocks of sum dt*F (this level as the fine side)
    int n_freg = 0;
    DevBuf<int64_t> coarse_off;  // [n_patches*6]: this level's leaf-patch faces next to refined patches
    DevBuf<double> creg;         // their [5][8][8] blocks of dt*F (this level as the coarse side)
    int n_creg = 0;
    DevBuf<int64_t> fix_list;    // [n_fix][13]: patch, coarse blocks[6], fine blocks[6]
    int n_fix = 0;
    DevBuf<int32_t> restrict_list;  // [n_restrict][2]: refined patch, child group
    int n_restrict = 0;
    bool bound = false;          // capacity arrays registered (levels >= 1)
    int32_t *w_corner = nullptr, *w_sib = nullptr, *w_parent = nullptr, *w_child = nullptr;
    double dt_prev = -1.0;       // last step size (W-cycle)
    double dt_last = 0.0;        // dt argument of the level's last step (< 0: the device's CFL dt)
    DevBuf<double> freg_save;    // fine registers before a step that may be retried
    int scal0 = 0;  // first of this level's 8 scalar slots
    int ring = 0;   // ring position of the newest state
    bool speed_valid = false;
    bool uniform = false;  // level 0 holding the whole root grid in the order of amr_hydro_uniform_tables
    // device-side bookkeeping (regrid_dev.cu): dense patch-position -> slot
    // map, ghost-position bits and ranks of the neighbour plan
    DevBuf<int32_t> posmap, gbits, grank;
    bool posmap_valid = false;
    bool host_stale = false;       // host table mirrors behind the device tables (refresh_host_tables)
    unsigned long long version = 0;       // bumped whenever the level's cell data change
    unsigned long long plan_version = 0;  // bumped whenever its neighbour plan changes
    // the coarse-fine ghost patches hold the interpolation at ghost_t of the
    // coarse level's data version ghost_cver under plan ghost_pver
    bool ghost_valid = false;
    cudaGraphExec_t gexec = nullptr;  // the level step as a CUDA graph (refined hierarchies)
    double ghost_t = 0.0;
    unsigned long long ghost_cver = 0, ghost_pver = 0;
    void release() {
        nbr.release();
        ustar.release();
        runs.release();
        run_off.release();
        n_runs = 0;
        chain_up.release();
        chain_len.release();
        work.release();
        has_work = false;
        ghost.release();
        ghost_info.release();
        ghost_ustar.release();
        ghost_nbr.release();
        ghost_S.release();
        phi[0].release();
        phi[1].release();
        gacc[0].release();
        gacc[1].release();
        ghost_acc.release();
        gc = 0;
        fine_off.release();
        freg.release();
        coarse_off.release();
        creg.release();
        freg_save.release();
        fix_list.release();
        restrict_list.release();
        posmap.release();
        gbits.release();
        grank.release();
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        posmap_valid = ghost_valid = false;
        n_patches = n_groups = 0;
    }
};

struct Box {
    int n = 0, n_groups = 0;
    double *U[2] = {nullptr, nullptr};
    double *S[2] = {nullptr, nullptr};  // dual-energy entropy fields
    int cur = 0;
    int ring = 0;
    bool speed_valid = false;
    DevBuf<int32_t> nbr;
    DevBuf<double> ustar;  // VL half-step state
    void release() {
        nbr.release();
        ustar.release();
        n = 0;
    }
};

// Launch configuration of the box-batch kernel chosen by the autotuner.
struct BoxTune {
    int grid = 0;        // CTAs of the persistent launch
    int chunked = 0;     // contiguous runs of work items per CTA (1) or grid-stride (0)
    int interleave = 0;  // work list interleaves the boxes (1) or is box-major (0)
    float ms = 0.f;      // measured time of one batch step
};

}  // namespace amrh

namespace amrh {
// Scratch of the device-side regrid (regrid_dev.cu): counts and error word
// (device, with a pinned host copy), prefix-sum block sums, selection and
// numbering arrays, the new level's tables before they replace the old ones,
// and the register-map flags and ranks.
struct RegridScratch {
    DevBuf<int32_t> cnt, bsum, keep, mark, rank, gnew, gpar;
    DevBuf<int32_t> corner, sib, parent, child, old_of, info, new_of;
    DevBuf<int32_t> cf_a, cf_b, cf_c, cf_d, cf_e, cf_f, cf_g, cf_h;
    DevBuf<int32_t> run_down, run_cnt, run_lpos, run_rpos, run_hist;  // z-runs of a plan
    DevBuf<int32_t> taken, frank, flist, mflag, mrank, nflag;  // group numbering with slots kept in place
    int32_t *hcnt = nullptr;  // pinned, 32 entries
    double *htime = nullptr;  // pinned, 8 entries: a time record (0..2), min_dt's reads (4, 5)
    void release() {
        for (DevBuf<int32_t> *b : {&cnt, &bsum, &keep, &mark, &rank, &gnew, &gpar, &corner, &sib, &parent, &child,
                                   &old_of, &info, &new_of, &cf_a, &cf_b, &cf_c, &cf_d, &cf_e, &cf_f, &cf_g, &cf_h,
                                   &run_down, &run_cnt, &run_lpos, &run_rpos, &run_hist, &taken, &frank,
                                   &flist, &mflag, &mrank, &nflag})
            b->release();
        if (hcnt) cudaFreeHost(hcnt);
        if (htime) cudaFreeHost(htime);
        hcnt = nullptr;
        htime = nullptr;
    }
};
}  // namespace amrh

struct amr_hydro_ctx {
    amr_hydro_params prm;
    cudaStream_t stream = nullptr;
    int device = 0, n_sm = 148, step_bps = 1;
    amrh::Level lv[amrh::MAX_LEVELS];
    amrh::Box boxes[amrh::MAX_BOXES];
    amrh::DevBuf<unsigned long long> scal;
    amrh::DevBuf<double> dtbuf;
    amrh::DevBuf<uint8_t> pflag;         // refinement flag scratch
    amrh::DevBuf<uint32_t> flag_summary;  // per-patch summary of where flagged cells lie
    amrh::DevBuf<double> psum;           // per-patch conservation partials
    amrh::RegridScratch rg;              // the device-side regrid's scratch
    amrh::DevBuf<double> adjbuf;         // dense scratch of the adjoint step
    // batched-box launch plan, tuning and its captured graph
    amrh::DevBuf<int32_t> box_plan;   // (box, group) work items
    amrh::DevBuf<uint8_t> box_desc;
    std::vector<int> plan_key, tune_key;
    amrh::BoxTune tune;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<long long> graph_key;
    // host-streamed steps (amr_hydro_advance_host): copy streams, per-slab
    // events and the dense device staging of the input and output states
    cudaStream_t xfer[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> slab_ev;
    amrh::DevBuf<double> hstage[2];
    // cells the step left unphysical, for the cell remedies (params.fallback)
    amrh::DevBuf<int64_t> fb_list;
    amrh::DevBuf<unsigned long long> fb_count;
    // self-gravity in the W-cycle (amr_hydro_set_gravity)
    bool shared_dt = false;  // shared time-step integration of the W-cycle
    double shared_step = 0.0;
    bool grav_on = false;
    double grav_G = 0.0, grav_omega = 1.7;
    int grav_iters = 60, grav_order = 2;
    // phase timing (amr_hydro_phase_timing): event pairs of the recorded
    // phases, spare events, and the nesting depth of the open phase scopes
    bool timing = false;
    int phase_depth = 0;
    struct PhaseRec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<PhaseRec> phase_recs;
    std::vector<cudaEvent_t> phase_spare;
    // root-level Poisson solver (fft.cu): the real grid, its half spectrum,
    // the twiddle tables (x, y, z) and, with isolated boundaries, the
    // transformed kernel
    amrh::DevBuf<double> fft_real, fft_cplx, fft_green;
    amrh::DevBuf<double> fft_tw;
    int fft_tw_n[3] = {0, 0, 0};
    bool fft_green_ready = false;
};

namespace amrh {
const char *status_str(amr_status s);
amr_status cuda_fail(cudaError_t e, const char *where);
double level_dh(const amr_hydro_ctx *c, int level);
amr_status level_speed(amr_hydro_ctx *c, int level);
size_t step_smem_bytes(int prec);
void scheme_stages(int scheme, int recon, int dual_energy, int &lo, int &hi);
void release_poisson(amr_hydro_ctx *c);
amr_status advance_once(amr_hydro_ctx *c, int level, double dt, int64_t *n_unphysical_out, const double *acc_n,
                        double c_acc = 0.0);
// Eq. (acc) as a signal speed: max over acc's values of (cfl / c_acc) sqrt(dh |a|)
// into *smax, so that cfl dh / *smax is the smaller of the two time steps.
amr_status launch_acc_speed(amr_hydro_ctx *c, const double *acc, int64_t n_values, double dh, double c_acc,
                            unsigned long long *smax);
struct StepParams;
amr_status launch_step(amr_hydro_ctx *c, const StepParams &P, int grid);
amr_status launch_step_raw(int prec, const StepParams &P, cudaStream_t stream);
amr_status launch_cell_remedies(amr_hydro_ctx *c, const StepParams &P, const double *base, int cfl1,
                                cudaStream_t s);
constexpr int64_t FB_CAP = 1 << 20;  // listed cells per step launch (more are counted unphysical)
// the VL predictor's half step on a level's coarse-fine ghost patches (vl_ghost.cu)
amr_status launch_vl_ghost_pred(amr_hydro_ctx *c, int level, const StepParams &P);
amr_status launch_max_speed(int prec, const double *U, int64_t n_slots, double gamma, int cfl1,
                            unsigned long long *smax, unsigned long long *nbad, int n_sm, cudaStream_t stream);
// AMR (amr_ops.cu, regrid.cpp)
amr_status fill_ghost_impl(amr_hydro_ctx *c, int level, double t);
amr_status interp_new_patches(amr_hydro_ctx *c, int coarse, double *out, const int32_t *out_slot,
                              const int32_t *info, int n_jobs, double *out_S = nullptr);
amr_status copy_slots(amr_hydro_ctx *c, double *dst, const double *src, const int32_t *map, int n,
                      int width = PSLOT_DOUBLES);
amr_status patch_flags_dev(amr_hydro_ctx *c, int level, uint8_t *pflag);
amr_status plan_level(amr_hydro_ctx *c, int level);
amr_status rebuild_cf(amr_hydro_ctx *c, int fine_level);
// self-gravity in the W-cycle (grav_amr.cu)
amr_status gravity_level_step(amr_hydro_ctx *c, int level, double dt);
amr_status gravity_solve_level(amr_hydro_ctx *c, int level);
amr_status fill_ghost_acc(amr_hydro_ctx *c, int level, double t);
amr_status launch_grav_correct(amr_hydro_ctx *c, int level, double dt, const double *acc_n, const double *acc_new);
// device-side bookkeeping (regrid_dev.cu)
amr_status regrid_dev(amr_hydro_ctx *c, int level);
amr_status build_posmap(amr_hydro_ctx *c, int level);
amr_status refresh_host_tables(amr_hydro_ctx *c, int level);
amr_status level_time(amr_hydro_ctx *c, int level);
// host planning (host_plan.cpp)
amr_status build_uniform_tables(const int np[3], int32_t *corner, int32_t *sib, int32_t *parent,
                                int32_t *child);
amr_status build_nbr_plan(int level, int n_patches, const int32_t *corner, const int32_t *sib,
                          const int32_t *parent, const int level_cells[3],
                          std::vector<int32_t> &nbr, std::vector<GhostInfo> &ghosts, int ghost_depth = 2,
                          bool corners = false);
// z-chains of a level's groups (same-level groups stacked in z), their
// runs of at most max_len groups, and the run length for a grid (host_plan.cpp).
void z_chains(int n_groups, const int32_t *nbr, std::vector<int32_t> &chains, std::vector<int32_t> &chain_off);
void cut_runs(const std::vector<int32_t> &chains, const std::vector<int32_t> &chain_off, int max_len,
              std::vector<int32_t> &runs, std::vector<int32_t> &run_off);
void build_runs(int n_groups, const int32_t *nbr, int max_len, std::vector<int32_t> &runs,
                std::vector<int32_t> &run_off);
int choose_run_len(const std::vector<int32_t> &chain_off, int grid, double e);

// A phase of the level path timed by an event pair on the context's stream
// (outermost scope only); does nothing while timing is off.
struct PhaseScope {
    amr_hydro_ctx *c;
    int phase;
    bool on = false;
    cudaEvent_t a = nullptr;
    PhaseScope(amr_hydro_ctx *ctx, int ph);
    ~PhaseScope();
};

// Kernel attributes set by cudaFuncSetAttribute hold per device: fn() runs
// once for each device it is first needed on (the current one), under a lock,
// so concurrent first calls from several host threads wait for one setter.
constexpr int MAX_DEVICES = 64;
struct DeviceOnce {
    std::mutex m;
    bool done[MAX_DEVICES] = {};
};
template <typename F>
amr_status once_per_device(DeviceOnce &o, F &&fn) {
    int dev = 0;
    amr_status st = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    if (dev < 0 || dev >= MAX_DEVICES) return AMR_E_INVAL;
    std::lock_guard<std::mutex> lock(o.m);
    if (o.done[dev]) return AMR_OK;
    if ((st = fn())) return st;
    o.done[dev] = true;
    return AMR_OK;
}
}  // namespace amrh

namespace amrh {
// Variables per coarse-fine flux register: the five conserved ones, and the
// dual-energy entropy's flux as a sixth.  A fine register block holds
// reg_vars x 16 x 16 doubles, a coarse one reg_vars x 8 x 8.
inline int reg_vars(const amr_hydro_ctx *c) { return c->prm.dual_energy ? 6 : 5; }
inline int64_t fine_block(const amr_hydro_ctx *c) { return 256 * (int64_t)reg_vars(c); }
inline int64_t coarse_block(const amr_hydro_ctx *c) { return 64 * (int64_t)reg_vars(c); }
}  // namespace amrh
