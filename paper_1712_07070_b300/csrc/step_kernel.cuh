// step_kernel.cuh -- the fused per-patch-group MUSCL-Hancock step
// (GAMER-2 section 2.2 scheme on section 3.1 patch groups; time step of
// section 2.6 Eq. CFL2 reduced on the fly).
//
// One CTA owns one patch group (2x2x2 patches = 16^3 cells) at a time and
// marches through its 20^3 ghosted tile plane by plane along z:
//   load   plane z+1 of the tile (gathered from the group's own 8 patches, its
//          56 same-level neighbours, or interpolated coarse-fine ghost
//          patches) and convert it to primitives in shared memory
//          (a ring of three planes);
//   B      limited slopes + Hancock half step for the cells of plane z whose
//          face states are needed (16x16 interior + the 64-cell ring of x/y
//          ghosts); x/y face states go to shared memory, the interior cell's
//          z face states stay in the owning thread's registers;
//   C      HLLC on the x and y faces of plane z and on the z face below it;
//   D      each thread finishes the update of its column's cell at z-1 and
//          starts the flux divergence of the cell at z.
// The 20^3 tile never exists in global memory (section 3.4: ghost zones are
// only allocated temporarily).
//
// The VL scheme (section 2.2) runs as two launches of the same march
// (STAGE): the predictor (ST_VL_PRED) keeps conserved cell averages in the
// ring, takes them as the face states of every cell and writes the half
// step U* = U^n - dt/(2 dh) sum_d (F_{d,+} - F_{d,-}); the corrector
// (ST_VL_CORR) reconstructs the limited piecewise-linear face states of U*
// (no Hancock increment) and updates U^n with their Riemann fluxes.
#pragma once
#include <type_traits>

#include "hydro_math.cuh"

namespace amrh {

constexpr int PS = 8;                 // patch edge
constexpr int PV = PS * PS * PS;      // cells per patch
constexpr int PSLOT = NV * PV;        // doubles per patch slot
constexpr int GE = 16;                // group edge
constexpr int TW = GE + 4;            // tile edge with 2 ghost cells per side (PLM)
constexpr int COLS = GE * GE;         // (x,y) columns of a group: one owner thread each
constexpr int MAX_WARPS = 8;

// Stage of the step a kernel instance computes.
constexpr int ST_MH = 0;       // MUSCL-Hancock step
constexpr int ST_VL_PRED = 1;  // VL half step U* from first-order fluxes of U^n
constexpr int ST_VL_CORR = 2;  // VL update of U^n with the fluxes of the PLM states of U*
constexpr int ST_CTU = 3;      // CTU step (ctu_kernel.cuh)
constexpr int ST_MH_PPM = 4;   // MUSCL-Hancock step with PPM reconstruction
constexpr int ST_CTU_PPM = 5;  // CTU step with PPM reconstruction
constexpr int ST_MH_DE = 6;    // MUSCL-Hancock step with the dual-energy formalism
constexpr int ST_MH_GRAV = 7;  // MUSCL-Hancock predictor of the gravity coupling
constexpr int ST_CTU_GRAV = 8;  // CTU (PLM) predictor of the gravity coupling
constexpr int N_STAGES = 9;
__host__ __device__ constexpr bool stage_ppm(int st) { return st == ST_MH_PPM || st == ST_CTU_PPM; }
__host__ __device__ constexpr bool stage_ctu(int st) {
    return st == ST_CTU || st == ST_CTU_PPM || st == ST_CTU_GRAV;
}

// Tile geometry for NG ghost cells per side (2: PLM, 3: PPM, whose face
// values reach two cells).  Rows y = -NG .. 15+NG; columns are staged in
// 16-byte x-pairs starting on even x, so the stored row runs from x = -OX
// (NG rounded up to even) to 15 + OX.  The ring keeps NR = 2 S + 1 planes for
// a stencil of half-width S = NG - 1 along z.
template <int NG>
struct Tile {
    static constexpr int S = NG - 1;
    static constexpr int NR = 2 * S + 1;
    static constexpr int OY = NG, OX = NG + (NG & 1);
    static constexpr int TY = GE + 2 * OY, TX = GE + 2 * OX;
    static constexpr int PAIRS = TY * TX / 2;
    __host__ __device__ static constexpr int slot(int t) { return (t + 4 * NR) % NR; }  // ring slot of plane t >= -NG
};

// Threads per CTA: one per (x,y) column of the group.  The FP32 kernel is
// register-bounded for two resident CTAs per SM, the FP64 kernel for one (its
// FP64 pipe is the bound, not latency).
template <typename real>
struct StepCfg {
    static constexpr int NT = 256;
    static constexpr int MINB = sizeof(real) == sizeof(double) ? 1 : 2;  // resident CTAs/SM targeted
};

// Coarse-fine flux registers (section 2.2 fix-up).  Faces f = 0..5 are
// -x, +x, -y, +y, -z, +z.  Fine side: fine_off[g*6+f] >= 0 is the offset (in
// doubles) of a [NREG][16][16] block of this level's fine register buffer for
// group face f lying on a coarse-fine interface; every step adds dt * F of
// each fine boundary face into it.  Coarse side: coarse_off[slot*6+f] >= 0 is
// the offset of a [NREG][8][8] block of this level's coarse register buffer for
// a leaf patch face next to a refined patch; every step stores dt * F there.
// Block index (v, t2, t1) with t1 < t2 the two transverse dimensions.  NREG
// is 5, or 6 with dual energy (the entropy's flux in the sixth).
struct CFRegs {
    const int64_t *fine_off;    // [n_groups*6] or null
    double *fine_buf;
    const int64_t *coarse_off;  // [n_slots*6] or null
    double *coarse_buf;
};

struct StepParams {
    const double *__restrict__ U_old;   // the state reconstructed (U* in the VL corrector)
    double *__restrict__ U_new;
    const double *__restrict__ U_base;  // VL corrector: U^n, the state the fluxes update
    int stage;                          // ST_MH, ST_VL_PRED or ST_VL_CORR (selects the instance)
    const int32_t *__restrict__ nbr;  // [n_groups][64] source of each 4x4x4 patch position
    const double *__restrict__ ghost; // interpolated coarse-fine ghost patches
    const int32_t *__restrict__ work; // optional list of group ids (null: work0..work0+n_work-1)
    int n_work;
    int work0;
    // optional z-runs: work item i is the groups runs[run_off[i] .. run_off[i+1]),
    // each the same-level group directly above the previous one
    const int32_t *__restrict__ runs;
    const int32_t *__restrict__ run_off;
    double dt;                               // >= 0: time step from the host
    const unsigned long long *smax_in;       // dt < 0: dt = cfl*dh/smax_in
    double cfl, dh, gamma;
    int limiter, riemann;                    // amr_limiter / amr_riemann
    double theta;                            // generalized minmod coefficient
    int fallback;                            // remedy (i): the Roe solver checks its intermediate states
    // remedies (ii)-(iii): unphysical updated cells are appended (as their
    // offset of variable 0 in U_new) for the cell-remedy kernel; null: counted
    unsigned long long *fb_count;
    int64_t *fb_list;
    int64_t fb_cap;
    // dual energy (ST_MH_DE): the entropy per unit volume [slot][8^3] before
    // and after the step, and the threshold on E_the / E_kin
    const double *__restrict__ S_old;
    double *__restrict__ S_new;
    const double *__restrict__ ghost_S;  // the entropy of the coarse-fine ghost patches [ghost][8^3]
    double de_xi;
    // gravity predictor (ST_MH_GRAV): the acceleration at t^n, [slot][3][8^3],
    // and on refined levels that of the coarse-fine ghost patches [ghost][3][8^3]
    const double *__restrict__ acc_n;
    const double *__restrict__ ghost_acc;
    unsigned long long *smax_out;            // max signal speed of the new state (bits)
    unsigned long long *n_bad;               // count of unphysical new cells
    unsigned long long *clear2;              // two scalars the kernel zeroes for the next step
    double *time_rec;                        // device record {dt used, t_new, t_old}
    CFRegs cf;
};

template <typename real, int NG = 2>
struct StepSmem {
    using Geo = Tile<NG>;
    static constexpr bool DE = false;
    real W[Geo::NR][NV][Geo::TY][Geo::TX];  // primitive ring, planes z-S .. z+S
    real XS[2][NV][GE][GE + 2];  // x-/x+ face states, cells x=-1..16, rows y=0..15
    real YS[2][NV][GE + 2][GE];  // y-/y+ face states, cells y=-1..16, columns x=0..15
    real FX[NV][GE][GE + 1];     // x flux at face x-1/2, x=0..16
    real FY[NV][GE + 1][GE];     // y flux at face y-1/2, y=0..16
    alignas(16) double raw[NV][Geo::TY * Geo::TX];  // next tile plane in flight (cp.async), x-pairs owned per thread
    alignas(16) double uo[2][NV][COLS];   // each column's U^n one plane ahead of its update (cp.async)
    // per-group tables, two slots (group k of a run uses slot k & 1)
    int nbr[2][64];
    long long cfo[2][6];   // fine register blocks of the group's faces (-1: none)
    long long cco[2][48];  // coarse register blocks of its 8 patches' faces (-1: none)
    double red[MAX_WARPS];
    double dt;
};

// The MUSCL-Hancock march with the entropy scalar s = P / rho^(gamma-1) of the
// dual-energy formalism: q = s / rho rides along in its own ring, face
// values, fluxes and staging (the same layouts as the hydro variables'
// with one component).
template <typename real>
struct StepSmemDE : StepSmem<real, 2> {
    static constexpr bool DE = true;
    real Q[3][TW][TW];       // q ring
    real QX[2][GE][GE + 2];  // s on the x-/x+ faces after the Hancock step
    real QY[2][GE + 2][GE];
    real FQX[GE][GE + 1];    // scalar x flux at face x-1/2
    real FQY[GE + 1][GE];
    alignas(16) double raws[TW * TW];  // next tile plane of s in flight
    alignas(16) double uos[2][COLS];   // each column's s^n one plane ahead of its update
};

// dt * F into the registers of the face between cells a (low) and b (high)
// along D at flux value F (compute type), fine face coordinates (t1, t2) in
// 0..15 within the group; pa / pb: local patch indices (0..7) of the two
// cells in the groups of table slots sa / sb when they belong to the run
// (-1 otherwise); fo: the fine register block of the face (-1: none).
template <typename real, typename SM>
__device__ __forceinline__ void cf_register(const SM &S, const StepParams &P, double dt,
                                            const real F[NV], int D, int t1, int t2, int sa, int pa, int sb,
                                            int pb, long long fo, real fs = real(0)) {
    double Fd[NV];
    double fsd = 0.0;  // the dual-energy entropy's flux (SM::DE)
    if constexpr (SM::DE) {
        if constexpr (sizeof(real) == sizeof(double)) fsd = fs;
        else fsd = f2d_bits(fs);
    }
    const long long ca = pa >= 0 ? S.cco[sa][pa * 6 + 2 * D + 1] : -1;  // high face of the low cell's patch
    const long long cb = pb >= 0 ? S.cco[sb][pb * 6 + 2 * D] : -1;      // low face of the high cell's patch
    if (fo < 0 && ca < 0 && cb < 0) return;
#pragma unroll
    for (int v = 0; v < NV; v++) {
        if constexpr (sizeof(real) == sizeof(double)) Fd[v] = F[v];
        else Fd[v] = f2d_bits(F[v]);
    }
    if (fo >= 0) {
        double *b = P.cf.fine_buf + fo;
#pragma unroll
        for (int v = 0; v < NV; v++) b[(v * 16 + t2) * 16 + t1] += dt * Fd[v];
        if constexpr (SM::DE) b[(NV * 16 + t2) * 16 + t1] += dt * fsd;
    }
    const int c1 = t1 & 7, c2 = t2 & 7;
    if (ca >= 0) {
        double *b = P.cf.coarse_buf + ca;
#pragma unroll
        for (int v = 0; v < NV; v++) b[(v * 8 + c2) * 8 + c1] = dt * Fd[v];
        if constexpr (SM::DE) b[(NV * 8 + c2) * 8 + c1] = dt * fsd;
    }
    if (cb >= 0) {
        double *b = P.cf.coarse_buf + cb;
#pragma unroll
        for (int v = 0; v < NV; v++) b[(v * 8 + c2) * 8 + c1] = dt * Fd[v];
        if constexpr (SM::DE) b[(NV * 8 + c2) * 8 + c1] = dt * fsd;
    }
}

// The face solver through a face normal to a runtime direction D: the normal momentum is
// swapped into the x slot, the x-normal solver runs, and the flux is swapped
// back (register selects only), so lanes of one warp can serve different
// directions without diverging.
template <typename real>
__device__ __forceinline__ void hllc_dir(const real uL[NV], const real uR[NV], int D, real F[NV],
                                         const Gas<real> &g) {
    real a[NV], b[NV], f[NV];
    a[0] = uL[0];
    a[4] = uL[4];
    a[1] = D == 1 ? uL[2] : (D == 2 ? uL[3] : uL[1]);
    a[2] = D == 1 ? uL[1] : uL[2];
    a[3] = D == 2 ? uL[1] : uL[3];
    b[0] = uR[0];
    b[4] = uR[4];
    b[1] = D == 1 ? uR[2] : (D == 2 ? uR[3] : uR[1]);
    b[2] = D == 1 ? uR[1] : uR[2];
    b[3] = D == 2 ? uR[1] : uR[3];
    face_flux<0>(a, b, f, g);
    F[0] = f[0];
    F[4] = f[4];
    F[1] = D == 1 ? f[2] : (D == 2 ? f[3] : f[1]);
    F[2] = D == 1 ? f[1] : f[2];
    F[3] = D == 2 ? f[1] : f[3];
}

// Source pointer for patch position q (0..63) of the current group.
__device__ __forceinline__ const double *patch_src(const StepParams &P, int s) {
    if (s >= 0) return P.U_old + (int64_t)s * PSLOT;
    if (s <= -2) return P.ghost + (int64_t)(-2 - s) * PSLOT;
    return nullptr;
}

// An unphysical updated cell (offset base of its variable 0 in U_new): into
// the list of the cell-remedy kernel when there is one and it has room.
__device__ __forceinline__ bool fb_append(const StepParams &P, int64_t base) {
    if (!P.fb_list) return false;
    const unsigned long long k = atomicAdd(P.fb_count, 1ull);
    if ((int64_t)k >= P.fb_cap) return false;
    P.fb_list[k] = base;
    return true;
}

// Load tile plane tl (-2..17 within the group of table slot ts) into the
// ring slot of run plane tr and convert to primitives.
template <typename real, int STAGE, typename SM>
__device__ __forceinline__ void load_plane(SM &S, const StepParams &P, int ts, int tl, int tr,
                                           const Gas<real> &g) {
    using G = typename SM::Geo;
    const int slot = G::slot(tr);
    const int qz = (tl + PS) >> 3, lz = (tl + PS) & 7;
    for (int i = threadIdx.x; i < G::TY * G::TX; i += StepCfg<real>::NT) {
        const int ty = i / G::TX - G::OY, tx = i % G::TX - G::OX;
        const int qy = (ty + PS) >> 3, ly = (ty + PS) & 7;
        const int qx = (tx + PS) >> 3, lx = (tx + PS) & 7;
        const double *src = patch_src(P, S.nbr[ts][qx + 4 * qy + 16 * qz]);
        real u[NV], w[NV];
        if (src) {
            const int off = lz * 64 + ly * 8 + lx;
#pragma unroll
            for (int v = 0; v < NV; v++) u[v] = to_real<real>(__ldg(src + v * PV + off));
            if constexpr (STAGE == ST_VL_PRED) {  // the predictor keeps conserved averages
#pragma unroll
                for (int v = 0; v < NV; v++) w[v] = u[v];
            } else {
                u2w(u, w, g);
            }
        } else {  // a position no stencil reads (a tile corner): benign state
            w[0] = real(1); w[1] = w[2] = w[3] = real(0); w[4] = real(1);
        }
#pragma unroll
        for (int v = 0; v < NV; v++) S.W[slot][v][ty + G::OY][tx + G::OX] = w[v];
        if constexpr (SM::DE) {  // q = s / rho (coarse-fine ghost patches: their interpolated s)
            const int sl = S.nbr[ts][qx + 4 * qy + 16 * qz];
            const double *ss = sl >= 0 ? P.S_old + (int64_t)sl * PV
                                       : (sl <= -2 ? P.ghost_S + (int64_t)(-2 - sl) * PV : nullptr);
            S.Q[slot][ty + G::OY][tx + G::OX] =
                ss ? to_real<real>(__ldg(ss + lz * 64 + ly * 8 + lx)) / w[0] : real(1);
        }
    }
}

// Asynchronous copy of tile plane tz into S.raw in 16-byte pieces: tile
// columns are taken in x-pairs (tx, tx+1) with tx even, which never straddle a
// patch and start on a 16-byte boundary in both the patch slot and S.raw.
// Thread j copies and later converts pair j (and j + 256), so the copy needs
// no CTA barrier, only the thread's own cp.async wait.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename real, typename SM>
__device__ __forceinline__ void issue_plane(SM &S, const StepParams &P, int ts, int tl) {
    using G = typename SM::Geo;
    const int qz = (tl + PS) >> 3, lz = (tl + PS) & 7;
    for (int j = threadIdx.x; j < G::PAIRS; j += StepCfg<real>::NT) {
        const int ty = j / (G::TX / 2) - G::OY, tx = 2 * (j % (G::TX / 2)) - G::OX;
        const int qy = (ty + PS) >> 3, ly = (ty + PS) & 7;
        const int qx = (tx + PS) >> 3, lx = (tx + PS) & 7;
        const int sl = S.nbr[ts][qx + 4 * qy + 16 * qz];
        const double *src = patch_src(P, sl);
        if (src) {
            const int off = lz * 64 + ly * 8 + lx;
#pragma unroll
            for (int v = 0; v < NV; v++) cp_async16(&S.raw[v][2 * j], src + v * PV + off);
            if constexpr (SM::DE)
                cp_async16(&S.raws[2 * j], (sl >= 0 ? P.S_old + (int64_t)sl * PV : P.ghost_S + (int64_t)(-2 - sl) * PV) + off);
        }
    }
    cp_async_commit();
}

// Wait for this thread's copies of tile plane tl (group of table slot ts,
// run plane tr) and convert them to primitives into the ring (the CTA
// barrier before stage B publishes them); the VL predictor keeps them
// conserved.
template <typename real, int STAGE, typename SM>
__device__ __forceinline__ void finish_plane(SM &S, int ts, int tl, int tr, const Gas<real> &g) {
    using G = typename SM::Geo;
    cp_async_wait_all();
    const int slot = G::slot(tr);
    const int qz = (tl + PS) >> 3;
    for (int j = threadIdx.x; j < G::PAIRS; j += StepCfg<real>::NT) {
        const int ty = j / (G::TX / 2) - G::OY, tx = 2 * (j % (G::TX / 2)) - G::OX;
        const int qy = (ty + PS) >> 3, qx = (tx + PS) >> 3;
        real w[2][NV], q[2] = {real(1), real(1)};
        if (S.nbr[ts][qx + 4 * qy + 16 * qz] != -1) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                real u[NV];
#pragma unroll
                for (int v = 0; v < NV; v++) u[v] = to_real<real>(S.raw[v][2 * j + h]);
                if constexpr (STAGE == ST_VL_PRED) {
#pragma unroll
                    for (int v = 0; v < NV; v++) w[h][v] = u[v];
                } else {
                    const real ri = u2w(u, w[h], g);
                    if constexpr (SM::DE) q[h] = to_real<real>(S.raws[2 * j + h]) * ri;  // q = s / rho
                }
            }
        } else {  // a position no stencil reads (a tile corner): benign state
#pragma unroll
            for (int h = 0; h < 2; h++) {
                w[h][0] = real(1); w[h][1] = w[h][2] = w[h][3] = real(0); w[h][4] = real(1);
            }
        }
#pragma unroll
        for (int v = 0; v < NV; v++) {
            S.W[slot][v][ty + G::OY][tx + G::OX] = w[0][v];
            S.W[slot][v][ty + G::OY][tx + G::OX + 1] = w[1][v];
        }
        if constexpr (SM::DE) {
            S.Q[slot][ty + G::OY][tx + G::OX] = q[0];
            S.Q[slot][ty + G::OY][tx + G::OX + 1] = q[1];
        }
    }
}

// PPM face values (lo at i-1/2, hi at i+1/2) of cell i from the values q[0..4]
// of one primitive component at cells i-2 .. i+2 along a direction
// (Colella & Woodward 1984): interpolation with the selected limiter's
// slopes, then the monotonicity constraints (an extremum flattens the cell,
// a face that would overshoot moves to 3 W_i - 2 W_other).
template <typename real>
__device__ __forceinline__ void ppm_faces(const real q[5], const Gas<real> &g, real &lo, real &hi) {
    const real dm = real(2) * half_slope(q[1] - q[0], q[2] - q[1], g);
    const real d0 = real(2) * half_slope(q[2] - q[1], q[3] - q[2], g);
    const real dp = real(2) * half_slope(q[3] - q[2], q[4] - q[3], g);
    const real sixth = real(1.0 / 6.0);
    real l = real(0.5) * (q[1] + q[2]) - (d0 - dm) * sixth;
    real r = real(0.5) * (q[2] + q[3]) - (dp - d0) * sixth;
    const real c = q[2];
    if (le0((r - c) * (c - l))) {
        l = c;
        r = c;
    } else {
        const real d = r - l, m = real(6) * (c - real(0.5) * (l + r));
        const real dmv = d * m, dd = d * d;
        if (gt0(dmv - dd)) l = real(3) * c - real(2) * r;
        else if (gt0(-dd - dmv)) r = real(3) * c - real(2) * l;
    }
    lo = l;
    hi = r;
}

// Primitive face values (low, high) along D of tile cell (X, Y) (ring
// indices) on plane z: W -/+ dW/2 with the limiter's slope (PLM), or the PPM
// face values.
template <typename real, int D, bool PPM, typename SM>
__device__ __forceinline__ void face_values(const SM &S, int X, int Y, int z, const Gas<real> &g, real wm[NV],
                                            real wp[NV]) {
    using G = typename SM::Geo;
    constexpr int R = PPM ? 2 : 1;
    int sl[2 * R + 1];
#pragma unroll
    for (int k = -R; k <= R; k++) sl[k + R] = G::slot(z + (D == 2 ? k : 0));
#pragma unroll
    for (int v = 0; v < NV; v++) {
        real q[2 * R + 1];
#pragma unroll
        for (int k = -R; k <= R; k++)
            q[k + R] = D == 0 ? S.W[sl[R]][v][Y][X + k] : (D == 1 ? S.W[sl[R]][v][Y + k][X] : S.W[sl[k + R]][v][Y][X]);
        if constexpr (PPM) {
            ppm_faces(q, g, wm[v], wp[v]);
        } else {
            const real hs = half_slope(q[1] - q[0], q[2] - q[1], g);
            wm[v] = q[1] - hs;
            wp[v] = q[1] + hs;
        }
    }
}

// Face states of tile cell (x,y) on plane z: reconstructed (PLM or PPM) face
// states and the Hancock half step (ST_MH, ST_MH_PPM), the reconstructed
// states alone (ST_VL_CORR), or the cell's conserved average on every face
// (ST_VL_PRED).  uf[2d] / uf[2d+1]: conserved state on the low / high face along d.
// With the dual-energy scalar (SM::DE), us[f]: s on face f, rho_f q_f with
// PLM q, after the Hancock step with F_s = s v_n.  The gravity predictor
// (ST_MH_GRAV) adds (dt/2) (0, rho_f ga, m_f . ga) of each reconstructed face
// state, ga the cell's acceleration at t^n (dt_half = dt/2).
// only_dim >= 0: only the two face states along that dimension are wanted
// (a ghost-ring cell of the group, whose other faces no face solve reads).
template <typename real, int STAGE, typename SM>
__device__ __forceinline__ void hancock_cell(const SM &S, int x, int y, int z, real dtdh_half, const Gas<real> &g,
                                             real uf[6][NV], real us[6], const real ga[3] = nullptr,
                                             real dt_half = real(0), int only_dim = -1) {
    using G = typename SM::Geo;
    const int X = x + G::OX, Y = y + G::OY;
    if constexpr (STAGE == ST_VL_PRED) {
        const int s0 = G::slot(z);
#pragma unroll
        for (int f = 0; f < 6; f++)
#pragma unroll
            for (int v = 0; v < NV; v++) uf[f][v] = S.W[s0][v][Y][X];
    } else {
        constexpr bool ppm = stage_ppm(STAGE), hancock = STAGE != ST_VL_CORR;
        real inc[NV] = {real(0), real(0), real(0), real(0), real(0)};
        real incs = real(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            real wm[NV], wp[NV], fm[NV], fp[NV];
            if (d == 0) face_values<real, 0, ppm>(S, X, Y, z, g, wm, wp);
            if (d == 1) face_values<real, 1, ppm>(S, X, Y, z, g, wm, wp);
            if (d == 2) face_values<real, 2, ppm>(S, X, Y, z, g, wm, wp);
            if constexpr (SM::DE) {  // the entropy scalar: PLM q, s = rho_f q_f, F_s = s v_n
                const int s0 = G::slot(z);
                const real qc = S.Q[s0][Y][X];
                const real ql = d == 0 ? S.Q[s0][Y][X - 1] : (d == 1 ? S.Q[s0][Y - 1][X] : S.Q[G::slot(z - 1)][Y][X]);
                const real qh = d == 0 ? S.Q[s0][Y][X + 1] : (d == 1 ? S.Q[s0][Y + 1][X] : S.Q[G::slot(z + 1)][Y][X]);
                const real hq = half_slope(qc - ql, qh - qc, g);
                us[2 * d] = wm[0] * (qc - hq);
                us[2 * d + 1] = wp[0] * (qc + hq);
                incs += us[2 * d] * wm[1 + d] - us[2 * d + 1] * wp[1 + d];
            }
            w2u(wm, uf[2 * d], g);
            w2u(wp, uf[2 * d + 1], g);
            if constexpr (hancock) {
                if (d == 0) { phys_flux<0>(wm, uf[0], fm); phys_flux<0>(wp, uf[1], fp); }
                if (d == 1) { phys_flux<1>(wm, uf[2], fm); phys_flux<1>(wp, uf[3], fp); }
                if (d == 2) { phys_flux<2>(wm, uf[4], fm); phys_flux<2>(wp, uf[5], fp); }
#pragma unroll
                for (int v = 0; v < NV; v++) inc[v] += fm[v] - fp[v];
            }
        }
        if constexpr (STAGE == ST_MH_GRAV) {
#pragma unroll
            for (int f = 0; f < 6; f++) {
                if (only_dim >= 0 && (f >> 1) != only_dim) continue;
                real src[NV];
                src[0] = real(0);
                src[1] = uf[f][0] * ga[0];
                src[2] = uf[f][0] * ga[1];
                src[3] = uf[f][0] * ga[2];
                src[4] = uf[f][1] * ga[0] + uf[f][2] * ga[1] + uf[f][3] * ga[2];
#pragma unroll
                for (int v = 0; v < NV; v++) uf[f][v] = (uf[f][v] + dtdh_half * inc[v]) + dt_half * src[v];
            }
        } else if constexpr (hancock) {
#pragma unroll
            for (int f = 0; f < 6; f++) {
                if (only_dim >= 0 && (f >> 1) != only_dim) continue;
#pragma unroll
                for (int v = 0; v < NV; v++) uf[f][v] += dtdh_half * inc[v];
            }
        }
        if constexpr (SM::DE) {
#pragma unroll
            for (int f = 0; f < 6; f++) {
                if (only_dim >= 0 && (f >> 1) != only_dim) continue;
                us[f] += dtdh_half * incs;
            }
        }
    }
}

// The acceleration at t^n of tile cell (x, y, zl) of the group in table slot
// ts (gravity predictor).
template <typename real, typename SM>
__device__ __forceinline__ void grav_at(const SM &S, const StepParams &P, int ts, int x, int y, int zl, real ga[3]) {
    const int q = ((x + PS) >> 3) + 4 * ((y + PS) >> 3) + 16 * ((zl + PS) >> 3);
    const int sl = S.nbr[ts][q];
    const int off = ((zl + PS) & 7) * 64 + ((y + PS) & 7) * 8 + ((x + PS) & 7);
    // a same-level slot, or a coarse-fine ghost patch (refined levels: g^n
    // interpolated from the coarse level)
    const double *src = sl >= 0 ? P.acc_n + (int64_t)sl * 3 * PV
                                : (sl <= -2 && P.ghost_acc ? P.ghost_acc + (int64_t)(-2 - sl) * 3 * PV : nullptr);
#pragma unroll
    for (int d = 0; d < 3; d++) ga[d] = src ? to_real<real>(__ldg(src + d * PV + off)) : real(0);
}

// Flux of the dual-energy scalar through a face: the mass flux F_rho times
// q = s / rho of the upwind face state.
template <typename real>
__device__ __forceinline__ real scalar_flux(real frho, real sL, real rL, real sR, real rR) {
    return frho * (ge0(frho) ? sL * rcp_(rL) : sR * rcp_(rR));
}

// Stage C face evaluations of plane z (local plane zl of the group in table
// slot ts; cf: whether that group touches a coarse-fine register).  Thread
// (cx, cy) takes the x face x = cx - 1/2 of row cy and the y face
// y = cy - 1/2 of column cx; one warp also takes the group's high faces,
// x = 16 - 1/2 of the 16 rows (lanes 0..15) and y = 16 - 1/2 of the 16
// columns (lanes 16..31), in one divergence-free pass through hllc_dir.  The
// FP64 pipe charges a whole warp instruction however few lanes are active,
// so that pass costs one solver evaluation instead of two.
template <typename real, typename SM>
__device__ __forceinline__ void x_face(SM &S, const StepParams &P, double dt, int row, int col, int zl,
                                       int ts, bool cf, const Gas<real> &g) {
    real uL[NV], uR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) { uL[v] = S.XS[1][v][row][col]; uR[v] = S.XS[0][v][row][col + 1]; }
    face_flux<0>(uL, uR, F, g);
#pragma unroll
    for (int v = 0; v < NV; v++) S.FX[v][row][col] = F[v];
    real fs = real(0);
    if constexpr (SM::DE) {
        fs = scalar_flux(F[0], S.QX[1][row][col], uL[0], S.QX[0][row][col + 1], uR[0]);
        S.FQX[row][col] = fs;
    }
    if (cf && (col & 7) == 0) {  // a patch face: x = 0 (group boundary) or x = 8
        const int pr = (row >> 3) * 2 + (zl >> 3) * 4;
        cf_register(S, P, dt, F, 0, row, zl, ts, col == 0 ? -1 : pr, ts, pr + (col >> 3),
                    col == 0 ? S.cfo[ts][0] : -1LL, fs);
    }
}

template <typename real, typename SM>
__device__ __forceinline__ void y_face(SM &S, const StepParams &P, double dt, int r, int col, int zl,
                                       int ts, bool cf, const Gas<real> &g) {
    real uL[NV], uR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) { uL[v] = S.YS[1][v][r][col]; uR[v] = S.YS[0][v][r + 1][col]; }
    face_flux<1>(uL, uR, F, g);
#pragma unroll
    for (int v = 0; v < NV; v++) S.FY[v][r][col] = F[v];
    real fs = real(0);
    if constexpr (SM::DE) {
        fs = scalar_flux(F[0], S.QY[1][r][col], uL[0], S.QY[0][r + 1][col], uR[0]);
        S.FQY[r][col] = fs;
    }
    if (cf && (r & 7) == 0) {  // a patch face: y = 0 (group boundary) or y = 8
        const int pr = (col >> 3) + (zl >> 3) * 4;
        cf_register(S, P, dt, F, 1, col, zl, ts, r == 0 ? -1 : pr, ts, pr + 2 * (r >> 3),
                    r == 0 ? S.cfo[ts][2] : -1LL, fs);
    }
}

template <typename real, typename SM>
__device__ __forceinline__ void high_faces(SM &S, const StepParams &P, double dt, int lane, int zl,
                                           int ts, bool cf, const Gas<real> &g) {
    const int k = lane & 15, D = lane >> 4;
    real uL[NV], uR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
        uL[v] = D == 0 ? S.XS[1][v][k][GE] : S.YS[1][v][GE][k];
        uR[v] = D == 0 ? S.XS[0][v][k][GE + 1] : S.YS[0][v][GE + 1][k];
    }
    hllc_dir(uL, uR, D, F, g);
#pragma unroll
    for (int v = 0; v < NV; v++) {
        if (D == 0) S.FX[v][k][GE] = F[v];
        else S.FY[v][GE][k] = F[v];
    }
    real fs = real(0);
    if constexpr (SM::DE) {
        if (D == 0) {
            fs = scalar_flux(F[0], S.QX[1][k][GE], uL[0], S.QX[0][k][GE + 1], uR[0]);
            S.FQX[k][GE] = fs;
        } else {
            fs = scalar_flux(F[0], S.QY[1][GE][k], uL[0], S.QY[0][GE + 1][k], uR[0]);
            S.FQY[GE][k] = fs;
        }
    }
    if (cf) {
        const int pa = D == 0 ? 1 + (k >> 3) * 2 + (zl >> 3) * 4 : (k >> 3) + 2 + (zl >> 3) * 4;
        cf_register(S, P, dt, F, D, k, zl, ts, pa, ts, -1, S.cfo[ts][2 * D + 1], fs);
    }
}

// The z face below column (cx, cy) at run plane z (0..16 len): HLLC of the
// column's own face states (registers), plus the coarse-fine registers of
// patch faces.  The cell below is in run group ka, the one above in kb (the
// same group except at a group boundary, where ka = kb - 1: two same-level
// groups, so no fine register, but each side's coarse registers);
// cfm: bit s set when the group in table slot s touches a register.
// With dual energy (SM::DE) also the scalar's flux fzs from the entropy on
// the face's two sides (zps_prev below, zms above).
template <typename real, typename SM>
__device__ __forceinline__ void z_face(const SM &S, const StepParams &P, double dt, const real zp_prev[NV],
                                       const real zm[NV], int cx, int cy, int z, int len, unsigned cfm, real fz[NV],
                                       const Gas<real> &g, real zps_prev = real(0), real zms = real(0),
                                       real *fzs = nullptr) {
    face_flux<2>(zp_prev, zm, fz, g);
    real fs = real(0);
    if constexpr (SM::DE) {
        fs = scalar_flux(fz[0], zps_prev, zp_prev[0], zms, zm[0]);
        *fzs = fs;
    }
    if ((z & 7) == 0) {
        const bool bot = z == 0, top = z == GE * len;
        const int ka = bot ? 0 : (z - 1) >> 4, kb = top ? len - 1 : z >> 4;
        if ((cfm >> (ka & 1)) & 1u || (cfm >> (kb & 1)) & 1u) {
            const int pl = (cx >> 3) + 2 * (cy >> 3);
            const long long fo = bot ? S.cfo[0][4] : (top ? S.cfo[(len - 1) & 1][5] : -1LL);
            cf_register(S, P, dt, fz, 2, cx, cy, ka & 1, bot ? -1 : pl + 4 * (((z - 1) & 15) >> 3), kb & 1,
                        top ? -1 : pl + 4 * ((z & 15) >> 3), fo, fs);
        }
    }
}

// Step-kernel instance (MODE) for a limiter / Riemann solver choice.
__host__ __device__ inline int scheme_mode(int limiter, int riemann) {
    if (riemann == RS_EXACT) return 2;
    return (limiter != LIM_VANLEER || riemann != RS_HLLC) ? 1 : 0;
}

// The tables of group grp into table slot ts; returns (per thread) whether
// an entry this thread loaded names a coarse-fine register.
template <typename SM>
__device__ __forceinline__ bool load_tables(SM &S, const StepParams &P, int ts, int grp) {
    const int tid = threadIdx.x;
    bool has = false;
    if (tid < 64) S.nbr[ts][tid] = P.nbr[(int64_t)grp * 64 + tid];
    if (tid < 6) {
        const long long o = P.cf.fine_off ? P.cf.fine_off[(int64_t)grp * 6 + tid] : -1;
        S.cfo[ts][tid] = o;
        has = o >= 0;
    }
    if (tid >= 64 && tid < 112) {
        const int k = tid - 64;
        const long long o = P.cf.coarse_off ? P.cf.coarse_off[((int64_t)grp * 8 + k / 6) * 6 + k % 6] : -1;
        S.cco[ts][k] = o;
        has = o >= 0;
    }
    return has;
}

// Local plane of a run group at whose iteration the marches load the next
// group's tables: after the group's bottom face (plane 0) used the previous
// group's, and at least one barrier before the first staging of the next
// group's bottom plane (plane 12 for the CTU march with PPM, which stages
// four planes ahead).
constexpr int TABLE_ZL = 8;

// Group k of a run: runs[off + k], or the single group `first`.
__device__ __forceinline__ int run_group(const int32_t *runs, int off, int first, int k) {
    return runs ? __ldg(runs + off + k) : first;
}

// A run of len patch groups stacked in z (each the same-level group directly
// above the previous one; len = 1: one group): the whole fused step, as one
// continuous z-march through the run's 16 len planes, so the ghost planes two
// neighbouring groups share are loaded and advanced by the Hancock step once.
// Plane z of the run is local plane z - 16k of run group k.  The caller has
// set S.dt; smax_r / nbad accumulate the new state's largest signal speed and
// its unphysical cells.
template <typename real, int STAGE, typename SM>
__device__ __forceinline__ void step_run(SM &S, const StepParams &P, const int32_t *runs, int off,
                                         int first, int len, double dt, const Gas<real> &g, real &smax_r,
                                         unsigned &nbad) {
    static_assert(StepCfg<real>::NT == COLS, "one thread per (x,y) column");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cx = tid & 15, cy = tid >> 4;  // this thread's (x,y) column
    // the VL predictor advances by half a step
    const double dtdh = (STAGE == ST_VL_PRED ? 0.5 * dt : dt) / P.dh;
    const real dtdh_r = (real)dtdh;
    const double *__restrict__ ubase = STAGE == ST_VL_CORR ? P.U_base : P.U_old;
    const real dtdh_half = (real)(0.5 * dt / P.dh);
    const int Z = GE * len;
    // group ids: of the current run plane's group, of the one below it (for
    // stage D at a group boundary) and of the next one (fetched with its tables)
    int gcur = run_group(runs, off, first, 0), gprev = gcur, gnext = gcur;
    unsigned cfm = 0;  // bit s: the group in table slot s touches a coarse-fine register
    if (__syncthreads_or(load_tables(S, P, 0, gcur))) cfm = 1u;
    // iteration z (from -1) reads ring planes z - S .. z + S (S = 1 for PLM,
    // 2 for PPM): planes -1 - S .. S - 2 are gathered now, plane S - 1 is
    // staged, and the top of iteration z converts plane z + S and stages
    // plane z + S + 1
    constexpr int SZ = SM::Geo::S;
    for (int t = -1 - SZ; t <= SZ - 2; t++) load_plane<real, STAGE>(S, P, 0, t, t, g);
    issue_plane<real>(S, P, 0, SZ - 1);

    real zp_prev[NV];   // high z face state of this column's cell at z-1
    real acc[NV];       // flux divergence of this column's cell at z-1 (minus its top z flux)
#pragma unroll
    for (int v = 0; v < NV; v++) { zp_prev[v] = real(0); acc[v] = real(0); }
    // the dual-energy scalar's counterparts (SM::DE)
    real zps_prev = real(0), accs = real(0), fzs = real(0);

    for (int z = -1; z <= Z; z++) {
        {  // plane z+S is ready to convert, plane z+S+1 to stage
            const int t1 = z + SZ, k1 = t1 < 0 ? 0 : min(t1 >> 4, len - 1);
            finish_plane<real, STAGE>(S, k1 & 1, t1 - GE * k1, t1, g);
            const int t2 = z + SZ + 1;
            if (t2 <= Z + SZ) {
                const int k2 = min(t2 >> 4, len - 1);
                issue_plane<real>(S, P, k2 & 1, t2 - GE * k2);
            }
        }
        __syncthreads();
        const int kz = z < 0 ? 0 : min(z >> 4, len - 1), zl = z - GE * kz;  // run group and local plane of z
        if (zl == 0 && z > 0) {  // entering run group kz: its id was fetched with its tables
            gprev = gcur;
            gcur = gnext;
        }
        if (z >= 0 && z < Z && tid < COLS / 2) {
            // U^n of columns 2 tid, 2 tid + 1 at plane z (16-byte copies), for
            // their update in the next iteration.  Issued after the barrier: the
            // slot was last read by those columns' threads in the previous
            // iteration's stage D; the next finish_plane waits for it.
            const int64_t own = (int64_t)gcur * 8;
            const int px = (2 * tid) & 15, py = (2 * tid) >> 4;
            const double *src = ubase + (own + (px >> 3) + 2 * (py >> 3) + 4 * (zl >> 3)) * PSLOT +
                                (zl & 7) * 64 + (py & 7) * 8 + (px & 7);
#pragma unroll
            for (int v = 0; v < NV; v++) cp_async16(&S.uo[z & 1][v][2 * tid], src + v * PV);
            if constexpr (SM::DE)
                cp_async16(&S.uos[z & 1][2 * tid], P.S_old + (own + (px >> 3) + 2 * (py >> 3) + 4 * (zl >> 3)) * PV +
                                                       (zl & 7) * 64 + (py & 7) * 8 + (px & 7));
            cp_async_commit();
        }
        // the next run group's tables, into the slot group kz - 1 used last
        // at run plane 16 kz (its top face); first read when plane
        // 16 (kz + 1) is staged, at iteration 16 kz + 13 (PPM) or later
        const bool load_next = zl == TABLE_ZL && kz + 1 < len;
        bool has_next = false;
        if (load_next) {
            gnext = run_group(runs, off, first, kz + 1);
            has_next = load_tables(S, P, (kz + 1) & 1, gnext);
        }

        // ---- B: Hancock states of plane z
        real zm[NV], zp[NV], fz[NV];
        real zms = real(0), zps = real(0);  // the scalar on the column cell's z faces
        const real dt_half = (real)(0.5 * dt);
        {
            real uf[6][NV], us[6], ga[3];
            if constexpr (STAGE == ST_MH_GRAV) grav_at(S, P, kz & 1, cx, cy, zl, ga);
            hancock_cell<real, STAGE>(S, cx, cy, z, dtdh_half, g, uf, us, ga, dt_half);
#pragma unroll
            for (int v = 0; v < NV; v++) { zm[v] = uf[4][v]; zp[v] = uf[5][v]; }
            if constexpr (SM::DE) {
                zms = us[4];
                zps = us[5];
            }
            // Sub-partitions 2 and 3 (warp & 2) have no ghost-ring cells in this
            // stage: they take their z face here rather than in stage C.
            if ((warp & 2) && z >= 0) {
                z_face(S, P, dt, zp_prev, zm, cx, cy, z, len, cfm, fz, g, zps_prev, zms, &fzs);
            }
            if (z >= 0 && z < Z) {
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    S.XS[0][v][cy][cx + 1] = uf[0][v];
                    S.XS[1][v][cy][cx + 1] = uf[1][v];
                    S.YS[0][v][cy + 1][cx] = uf[2][v];
                    S.YS[1][v][cy + 1][cx] = uf[3][v];
                }
                if constexpr (SM::DE) {
                    S.QX[0][cy][cx + 1] = us[0];
                    S.QX[1][cy][cx + 1] = us[1];
                    S.QY[0][cy + 1][cx] = us[2];
                    S.QY[1][cy + 1][cx] = us[3];
                }
            }
        }
        if (z >= 0 && z < Z && tid < 64) {
            // ring cells: x = -1 / 16 (rows 0..15), then y = -1 / 16 (columns 0..15)
            const int r = tid & 15;
            const bool xring = tid < 32;
            const int side = (tid >> 4) & 1;
            const int x = xring ? (side ? GE : -1) : r;
            const int y = xring ? r : (side ? GE : -1);
            real uf[6][NV], us[6], ga[3];
            if constexpr (STAGE == ST_MH_GRAV) grav_at(S, P, kz & 1, x, y, zl, ga);
            hancock_cell<real, STAGE>(S, x, y, z, dtdh_half, g, uf, us, ga, dt_half, xring ? 0 : 1);
            if (xring) {
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    S.XS[0][v][y][x + 1] = uf[0][v];
                    S.XS[1][v][y][x + 1] = uf[1][v];
                }
                if constexpr (SM::DE) {
                    S.QX[0][y][x + 1] = us[0];
                    S.QX[1][y][x + 1] = us[1];
                }
            } else {
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    S.YS[0][v][y + 1][x] = uf[2][v];
                    S.YS[1][v][y + 1][x] = uf[3][v];
                }
                if constexpr (SM::DE) {
                    S.QY[0][y + 1][x] = us[2];
                    S.QY[1][y + 1][x] = us[3];
                }
            }
        }
        if (load_next) {  // uniform: every thread takes the same branch
            const unsigned bit = 1u << ((kz + 1) & 1);
            cfm = __syncthreads_or(has_next) ? (cfm | bit) : (cfm & ~bit);
        } else {
            __syncthreads();
        }

        // ---- C: the z face below the column (sub-partitions 0, 1), its x and
        // y faces, and the group's high faces on warp 2 (sub-partition 2), so
        // every sub-partition's FP64 share carries 5 or 6 face evaluations
        // here after 3 or 2 Hancock cells (+2 z faces) in stage B
        if (!(warp & 2) && z >= 0) {
            z_face(S, P, dt, zp_prev, zm, cx, cy, z, len, cfm, fz, g, zps_prev, zms, &fzs);
        }
        if (z >= 0 && z < Z) {
            const int ts = kz & 1;
            const bool cf = (cfm >> ts) & 1u;
            x_face(S, P, dt, cy, cx, zl, ts, cf, g);
            y_face(S, P, dt, cy, cx, zl, ts, cf, g);
            if (warp == 2) high_faces(S, P, dt, lane, zl, ts, cf, g);
        }
        __syncthreads();

        // ---- D: finish cell (cx,cy,z-1), start cell (cx,cy,z)
        if (z >= 1) {
            const int zc = z - 1, zcl = zc & (GE - 1);  // cell z-1: in the group below at a boundary
            const int64_t base = ((int64_t)(zl == 0 ? gprev : gcur) * 8 + (cx >> 3) + 2 * (cy >> 3) +
                                  4 * (zcl >> 3)) * PSLOT +
                                 (zcl & 7) * 64 + (cy & 7) * 8 + (cx & 7);
            real ur[NV];  // the new state in the compute type, for its signal speed
            double una[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const real tot = acc[v] + fz[v];
                const double uo = S.uo[zc & 1][v][tid];
                double un;
                if constexpr (sizeof(real) == sizeof(double)) {
                    un = uo - dtdh * tot;
                    ur[v] = un;
                } else {
                    // FP32 increment accumulated into the FP64 state
                    const real inc = dtdh_r * tot;
                    un = uo - f2d_bits(inc);
                    ur[v] = d2f_bits(uo) - inc;
                }
                if constexpr (SM::DE) una[v] = un;
                else P.U_new[base + v * PV] = un;
            }
            if constexpr (SM::DE) {
                // the scalar's update, then the dual-energy choice (FP64): E from
                // s where E_the < xi E_kin, else s from E
                const real tots = accs + fzs;
                const double so = S.uos[zc & 1][tid];
                double sn;
                if constexpr (sizeof(real) == sizeof(double)) sn = so - dtdh * tots;
                else sn = so - f2d_bits(dtdh_r * tots);
                const double ekin = 0.5 * (una[1] * una[1] + una[2] * una[2] + una[3] * una[3]) / una[0];
                const double eth = una[4] - ekin;
                // rho^(gamma-1) at the flux precision: an FP64 pow costs about as much
                // FP64 pipe time as the FP32 mode's whole cell update
                if constexpr (sizeof(real) == sizeof(double)) {
                    const double rg = pow(una[0], P.gamma - 1.0);
                    if (eth < P.de_xi * ekin) una[4] = ekin + sn * rg / (P.gamma - 1.0);
                    else sn = (P.gamma - 1.0) * eth / rg;
                } else {  // the choice itself stays in FP64
                    const float rg = powf((float)una[0], (float)(P.gamma - 1.0));
                    if (eth < P.de_xi * ekin) una[4] = ekin + sn * (double)(rg / (float)(P.gamma - 1.0));
                    else sn = eth * (double)((float)(P.gamma - 1.0) / rg);
                }
                P.S_new[base / PSLOT * PV + base % PSLOT] = sn;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    P.U_new[base + v * PV] = una[v];
                    ur[v] = to_real<real>(una[v]);
                }
            }
            if constexpr (STAGE != ST_VL_PRED) {
                bool ok;
                const real s = cfl_speed(ur, g, ok);
                if (!ok && !fb_append(P, base)) nbad++;
                if (s > smax_r) smax_r = s;
            }
        }
        if (z >= 0 && z < Z) {
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const real dxy = (S.FX[v][cy][cx + 1] - S.FX[v][cy][cx]) +
                                 (S.FY[v][cy + 1][cx] - S.FY[v][cy][cx]);
                acc[v] = dxy - fz[v];
            }
            if constexpr (SM::DE)
                accs = ((S.FQX[cy][cx + 1] - S.FQX[cy][cx]) + (S.FQY[cy + 1][cx] - S.FQY[cy][cx])) - fzs;
        }
#pragma unroll
        for (int v = 0; v < NV; v++) zp_prev[v] = zp[v];
        zps_prev = zps;
    }
    __syncthreads();  // the next run overwrites the tables and the ring
}

}  // namespace amrh

#include "ctu_kernel.cuh"

namespace amrh {

// Shared memory of a kernel instance's march.
template <typename real, int STAGE>
using StageSmem = std::conditional_t<
    STAGE == ST_MH_DE, StepSmemDE<real>,
    std::conditional_t<stage_ctu(STAGE), CtuSmem<real, stage_ppm(STAGE) ? 3 : 2>,
                       StepSmem<real, stage_ppm(STAGE) ? 3 : 2>>>;

// One run (or group) of the instance's march.
template <typename real, int STAGE>
__device__ __forceinline__ void stage_run(StageSmem<real, STAGE> &S, const StepParams &P, const int32_t *runs,
                                          int off, int first, int len, double dt, const Gas<real> &g, real &smax_r,
                                          unsigned &nbad) {
    if constexpr (stage_ctu(STAGE))
        ctu_run<real, STAGE == ST_CTU_GRAV>(S, P, runs, off, first, len, dt, g, smax_r, nbad);
    else step_run<real, STAGE>(S, P, runs, off, first, len, dt, g, smax_r, nbad);
}

// MODE 0: the default scheme (van Leer-type limiter, HLLC) as compile-time
// constants, so the scheme branches fold away; MODE 1: the limiter of P
// and its HLLC, HLLE or Roe solver; MODE 2: the limiter of P and the exact
// solver (kept out of the other instances: its Newton iteration is a call).
// STAGE: ST_MH, one of the two VL launches (the predictor reduces nothing:
// the corrector reduces the new state's signal speed), or ST_CTU.
template <typename real, int MODE, int STAGE>
__global__ void __launch_bounds__(StepCfg<real>::NT, StepCfg<real>::MINB) k_hydro_step(StepParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StageSmem<real, STAGE> &S = *reinterpret_cast<StageSmem<real, STAGE> *>(smem_raw);
    const int tid = threadIdx.x;

    Gas<real> g;
    g.gamma = (real)P.gamma;
    g.gm1 = (real)(P.gamma - 1.0);
    g.inv_gm1 = (real)(1.0 / (P.gamma - 1.0));
    if constexpr (MODE != 0) {
        g.lim = P.limiter;
        g.htheta = (real)(0.5 * P.theta);
    }
    if constexpr (MODE == 1)  // a value the compiler can see is never RS_EXACT
        g.rs = P.riemann == RS_HLLE ? RS_HLLE : (P.riemann == RS_ROE ? RS_ROE : RS_HLLC);
    g.fb = P.fallback;
    if constexpr (MODE == 2) g.rs = RS_EXACT;

    if (tid == 0) {
        double dt = P.dt;
        if (dt < 0.0) dt = P.cfl * P.dh / __longlong_as_double((long long)*P.smax_in);
        S.dt = dt;
        if (blockIdx.x == 0 && P.clear2) {
            // the slots the following step will accumulate into (its smax_out
            // and n_bad); nothing reads or writes them during this step
            P.clear2[0] = 0ull;
            P.clear2[3] = 0ull;
        }
        if (blockIdx.x == 0 && P.time_rec) {
            const double t = P.time_rec[1];
            P.time_rec[0] = dt;
            P.time_rec[2] = t;
            P.time_rec[1] = t + dt;
        }
    }
    __syncthreads();
    const double dt = S.dt;
    real smax_r = real(0);
    unsigned nbad = 0;

    for (int wi = blockIdx.x; wi < P.n_work; wi += gridDim.x) {
        if (P.run_off) {
            const int o = __ldg(P.run_off + wi);
            stage_run<real, STAGE>(S, P, P.runs, o, 0, __ldg(P.run_off + wi + 1) - o, dt, g, smax_r, nbad);
        } else {
            stage_run<real, STAGE>(S, P, (const int32_t *)nullptr, 0, P.work ? P.work[wi] : P.work0 + wi, 1, dt, g,
                                   smax_r, nbad);
        }
    }
    if constexpr (STAGE == ST_VL_PRED) return;

    // ---- block reduction of the signal speed, one atomic per block
    double smax = (double)smax_r;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    unsigned nb = nbad;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, o);
    if ((tid & 31) == 0) S.red[tid >> 5] = smax;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int i = 0; i < StepCfg<real>::NT / 32; i++) m = fmax(m, S.red[i]);
        // positive doubles order like their bit patterns: exact, order-free max
        atomicMax(P.smax_out, (unsigned long long)__double_as_longlong(m));
    }
    if ((tid & 31) == 0 && nb) atomicAdd(P.n_bad, (unsigned long long)nb);
}

// ---- independent periodic boxes in one persistent launch ------------------------

// A box registered with amr_hydro_set_box: a fully covered periodic level.
struct BoxDesc {
    double *U[2];
    double *S[2];                 // dual-energy entropy fields (null without dual energy)
    double *ustar;                // VL half-step state (null for MUSCL-Hancock)
    const int32_t *nbr;           // [n_groups][64]
    unsigned long long *scal;     // the box's 8 scalar slots (ring of speeds, counts)
    double dh;
    int n_groups, cur0, ring0, log_index;
};

struct BoxLaunch {
    const BoxDesc *desc;
    const int2 *work;   // (box, group) items
    int n_work;
    int step;           // step index within this batch: buffers and ring advance with it
    int chunked;        // 1: each CTA takes a contiguous run of items; 0: grid-stride
    double cfl, gamma;
    int limiter, riemann;  // amr_limiter / amr_riemann
    double theta;          // generalized minmod coefficient
    int fallback;          // remedies for unphysical results
    double dt_override; // >= 0 (autotuning): fixed dt, no logging
    double *dt_log;     // [steps][n_boxes] or null
    int n_boxes;
    double de_xi;       // dual energy (ST_MH_DE): the threshold on E_the / E_kin
};

// MODE 0: the default scheme (van Leer-type limiter, HLLC) as compile-time
// constants, so the scheme branches fold away; MODE 1: the limiter of B
// and its HLLC, HLLE or Roe solver; MODE 2: the limiter of B and the exact
// solver (kept out of the other instances: its Newton iteration is a call).
// STAGE: ST_MH, or one of the two VL launches of a step (the predictor
// writes each box's U*, logs and reduces nothing; both take the box's dt
// from the same speed slot).
template <typename real, int MODE, int STAGE>
__global__ void __launch_bounds__(StepCfg<real>::NT, StepCfg<real>::MINB) k_hydro_step_boxes(BoxLaunch B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StageSmem<real, STAGE> &S = *reinterpret_cast<StageSmem<real, STAGE> *>(smem_raw);
    const int tid = threadIdx.x;
    Gas<real> g;
    g.gamma = (real)B.gamma;
    g.gm1 = (real)(B.gamma - 1.0);
    g.inv_gm1 = (real)(1.0 / (B.gamma - 1.0));
    if constexpr (MODE != 0) {
        g.lim = B.limiter;
        g.htheta = (real)(0.5 * B.theta);
    }
    if constexpr (MODE == 1)  // a value the compiler can see is never RS_EXACT
        g.rs = B.riemann == RS_HLLE ? RS_HLLE : (B.riemann == RS_ROE ? RS_ROE : RS_HLLC);
    g.fb = B.fallback;
    if constexpr (MODE == 2) g.rs = RS_EXACT;
    int first, last, stride;
    if (B.chunked) {
        const int per = (B.n_work + gridDim.x - 1) / gridDim.x;
        first = blockIdx.x * per;
        last = min(B.n_work, first + per);
        stride = 1;
    } else {
        first = blockIdx.x;
        last = B.n_work;
        stride = gridDim.x;
    }
    for (int wi = first; wi < last; wi += stride) {
        const int2 it = B.work[wi];
        const BoxDesc &d = B.desc[it.x];
        const int cur = (d.cur0 + B.step) & 1;
        const int r_in = (d.ring0 + B.step) % 3, r_out = (d.ring0 + B.step + 1) % 3, r_clr = (d.ring0 + B.step + 2) % 3;
        if (tid == 0) {
            double dt = B.dt_override;
            if (dt < 0.0) dt = B.cfl * d.dh / __longlong_as_double((long long)d.scal[r_in]);
            S.dt = dt;
            if (STAGE != ST_VL_PRED && it.y == 0 && B.dt_override < 0.0) {
                d.scal[r_clr] = 0ull;
                d.scal[3 + r_clr] = 0ull;
                if (B.dt_log) B.dt_log[(int64_t)B.step * B.n_boxes + d.log_index] = dt;
            }
        }
        __syncthreads();
        StepParams P;
        P.U_old = STAGE == ST_VL_CORR ? d.ustar : d.U[cur];
        P.U_new = STAGE == ST_VL_PRED ? d.ustar : d.U[1 - cur];
        P.U_base = d.U[cur];
        P.S_old = d.S[cur];
        P.S_new = d.S[1 - cur];
        P.de_xi = B.de_xi;
        P.stage = STAGE;
        P.fallback = B.fallback;
        P.nbr = d.nbr;
        P.ghost = nullptr;
        P.work = nullptr;
        P.n_work = d.n_groups;
        P.dt = S.dt;
        P.smax_in = nullptr;
        P.cfl = B.cfl;
        P.dh = d.dh;
        P.gamma = B.gamma;
        P.smax_out = d.scal + r_out;
        P.n_bad = d.scal + 3 + r_out;
        P.clear2 = nullptr;
        P.time_rec = nullptr;
        P.fb_count = nullptr;  // the box batch counts unphysical cells (no cell remedies)
        P.fb_list = nullptr;
        P.fb_cap = 0;
        P.cf.fine_off = nullptr;
        P.cf.fine_buf = nullptr;
        P.cf.coarse_off = nullptr;
        P.cf.coarse_buf = nullptr;
        real smax_r = real(0);
        unsigned nbad = 0;
        stage_run<real, STAGE>(S, P, (const int32_t *)nullptr, 0, it.y, 1, S.dt, g, smax_r, nbad);
        if constexpr (STAGE == ST_VL_PRED) continue;  // step_run ends with a CTA barrier
        // this group's largest signal speed and unphysical count into its box
        double smax = (double)smax_r;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        unsigned nb = nbad;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, o);
        if ((tid & 31) == 0) S.red[tid >> 5] = smax;
        __syncthreads();
        if (tid == 0) {
            double m = 0.0;
            for (int i = 0; i < StepCfg<real>::NT / 32; i++) m = fmax(m, S.red[i]);
            atomicMax(P.smax_out, (unsigned long long)__double_as_longlong(m));
        }
        if ((tid & 31) == 0 && nb) atomicAdd(P.n_bad, (unsigned long long)nb);
        __syncthreads();
    }
}

}  // namespace amrh
