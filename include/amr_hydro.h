/*
 * amr_hydro.h -- C ABI of the B300-native GAMER-2 patch-group hydro update.
 *
 * The method (GAMER-2, Schive et al. 2018):
 *   - section 2.1: block-structured AMR of fixed 8^3-cell patches, refinement
 *     ratio 2, a patch has 0 or 8 children and up to 26 siblings; patch
 *     groups of 2x2x2 sibling patches are the unit of hydro work (section
 *     3.1); adaptive per-level time steps advanced as a W-cycle.
 *   - section 2.2: MUSCL-Hancock (MHM) with PLM on primitive variables, a
 *     van Leer-type limiter and the HLLC Riemann solver; after a coarse
 *     level synchronises with its child level, restriction (volume-weighted
 *     average of the children) and the coarse-fine flux fix-up.
 *   - section 2.6: time step of Eq. (CFL2),
 *     dt = C_CFL dh / max(|vx|+|vy|+|vz|+3 c_s).
 *
 * Conventions for every entry point:
 *   - Ownership: the caller owns every state and table array; the library
 *     borrows raw device pointers and never frees them.  The context owns
 *     only its scratch (neighbour plans, interpolated coarse-fine ghost
 *     patches, coarse-fine flux registers, reduction scalars).
 *   - Layout of a level's state: U[slot][var][z][y][x] in FP64, 8^3 cells per
 *     slot, vars (rho, rho vx, rho vy, rho vz, E), x fastest.  Patch group g
 *     owns slots 8g..8g+7 in local order x fastest, then y, then z.
 *   - Streams: every call is asynchronous on the context's CUDA stream unless
 *     it returns a host value (min_dt to a host pointer, conserved_sum,
 *     advance_level with a non-NULL n_unphysical_out), which synchronises
 *     that stream.
 *   - Errors: every call returns an amr_status; kernels never trap.  Invalid
 *     arguments are rejected before any launch.
 *   - Threading: a context is used by one host thread at a time.
 */
#ifndef AMR_HYDRO_H
#define AMR_HYDRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMR_OK = 0,
    AMR_E_INVAL = 1,      /* bad argument (null pointer, size, level, ...) */
    AMR_E_NOMEM = 2,      /* device or host allocation failed */
    AMR_E_CUDA = 3,       /* a CUDA runtime call failed */
    AMR_E_UNPHYSICAL = 4, /* rho<=0 or P<=0 in the updated state */
    AMR_E_TIMEOUT = 5,    /* a bounded device wait ran out */
    AMR_E_NESTING = 6     /* the hierarchy violates proper nesting */
} amr_status;

typedef enum {
    AMR_FP64 = 0,       /* every step of the update in IEEE FP64 */
    AMR_FP32_ACC64 = 1  /* reconstruction, Hancock step and HLLC in FP32;
                           conserved-variable accumulation, flux fix-up,
                           dt and conservation reductions in FP64 */
} amr_precision;

/* Slope limiter of the piecewise-linear reconstruction (section 2.2 lists
 * these; definitions after Toro 2009).  With a = W_i - W_{i-1} and
 * b = W_{i+1} - W_i per primitive component, every limiter is 0 unless ab > 0. */
typedef enum {
    AMR_LIM_VANLEER = 0,    /* van Leer-type 2ab/(a+b) (the default) */
    AMR_LIM_GMINMOD = 1,    /* generalized minmod sign(a) min(t|a|, |a+b|/2, t|b|), t = minmod_coeff */
    AMR_LIM_ALBADA = 2,     /* van Albada-type ab(a+b)/(a^2+b^2) */
    AMR_LIM_VL_GMINMOD = 3  /* hybrid: the smaller in magnitude of the van Leer-type and
                               generalized minmod slopes */
} amr_limiter;

/* Riemann solver at every cell face (section 2.2). */
typedef enum {
    AMR_RS_HLLC = 0,  /* HLLC, Einfeldt/Roe outer speeds (the default) */
    AMR_RS_HLLE = 1,  /* HLLE (Einfeldt 1991) with the same outer speeds */
    AMR_RS_ROE = 2,   /* Roe (1981), Harten-Hyman entropy fix on the acoustic waves */
    AMR_RS_EXACT = 3  /* exact solver (Newton on the star pressure): Godunov flux at x/t = 0 */
} amr_riemann;

/* Integration scheme of the hydro step (section 2.2). */
typedef enum {
    AMR_SCHEME_MH = 0, /* MUSCL-Hancock: data-reconstructed half step (the default) */
    AMR_SCHEME_VL = 1, /* VL: half step U* = U^n - dt/(2 dh) sum_d (F_{d,+} - F_{d,-}) from the
                          Riemann fluxes of the cell averages, then the Riemann fluxes of the
                          limited piecewise-linear face states of U* update U^n.  Single-level
                          grids only: uniform levels (lmax = 0) and the batched boxes. */
    AMR_SCHEME_CTU = 2 /* CTU (Colella 1990), six Riemann solves per cell: face states along d
                          advanced by dt/2 with d's own flux difference, first fluxes, a
                          transverse correction -(dt/2dh) of the cell's first-flux differences
                          along the other two directions, final fluxes.  Time step of
                          Eq. (CFL1), C_CFL <= 0.5. */
} amr_scheme;

/* Reconstruction of the face states (section 2.2), on primitive variables. */
typedef enum {
    AMR_RECON_PLM = 0, /* piecewise linear with the selected limiter (the default) */
    AMR_RECON_PPM = 1  /* piecewise parabolic (Colella & Woodward 1984): face values
                          (W_i + W_{i+1})/2 - (dW_{i+1} - dW_i)/6 from the limiter's slopes,
                          then the CW84 monotonicity constraints; three ghost cells.
                          With AMR_SCHEME_MH and AMR_SCHEME_CTU. */
} amr_recon;

/* Boundary condition of the root-level gravity solve (section 2.3). */
typedef enum {
    AMR_GRAVITY_PERIODIC = 0, /* the 7-point Laplacian's Green's function on the periodic box */
    AMR_GRAVITY_ISOLATED = 1  /* every cell a point mass rho dh^3 at its centre, the potential the
                                 pairwise sum -G sum_{j != i} m_j / |r_i - r_j| (zero-padded FFT
                                 convolution on a grid of at least 2 N + 4 cells per axis) */
} amr_gravity_bc;

/* Run parameters (section 2.1 and 2.6 symbols). */
typedef struct {
    double gamma;        /* adiabatic index */
    double cfl;          /* C_CFL of Eq. (CFL2) */
    double c_inc, c_dec; /* dt increase / decrease fractions of section 2.1 */
    double theta;        /* refinement threshold (normalised density gradient) */
    int lmax;            /* maximum refinement level (0..7) */
    int nbuf[8];         /* flag-buffer width N_buf per level (section 2.1) */
    int prec;            /* amr_precision */
    int periodic[3];     /* 1 = periodic along x, y, z (only periodic is built) */
    double box[3];       /* domain edge lengths; cells are cubic */
    int root_n[3];       /* root-level cells per dimension, multiples of 16 */
    int max_patches;     /* slot capacity per level, a multiple of 8 */
    int limiter;         /* amr_limiter (0: van Leer-type) */
    int riemann;         /* amr_riemann (0: HLLC) */
    double minmod_coeff; /* generalized minmod coefficient in [1, 2]; 0 means 1.5 */
    int scheme;          /* amr_scheme (0: MUSCL-Hancock); AMR_SCHEME_VL needs lmax = 0; the
                            dt of AMR_SCHEME_CTU follows Eq. (CFL1), of the others Eq. (CFL2) */
    int recon;           /* amr_recon (0: PLM); PPM not with AMR_SCHEME_VL */
    int fallback;        /* 1: remedies for unphysical results (section 2.2): the Roe solver
                            falls back to HLLE where an intermediate state has rho <= 0 or
                            P <= 0; an unphysical updated cell is recomputed first order
                            unsplit from U^n, then first order dimensionally split */
    double dt_min;       /* > 0: a level step that leaves unphysical cells is recomputed with
                            dt x 0.8 until it succeeds or dt < dt_min (AMR_E_UNPHYSICAL);
                            0: no retry */
    int dual_energy;     /* 1: the dual-energy formalism (section 2.2) on single-level grids,
                            refined hierarchies (the entropy is interpolated, flux-registered,
                            fixed up and restricted like the conserved variables) and in the
                            box batch, with MUSCL-Hancock + PLM: the entropy per unit volume
                            s = P / rho^(gamma-1) (arrays of amr_hydro_set_entropy) is carried
                            as a passive scalar (PLM q = s / rho, F_s = mass flux x upwind q);
                            after the update E = E_kin + s rho^(gamma-1)/(gamma-1) where
                            E_the < dual_xi E_kin, else s is reset from E */
    double dual_xi;      /* the threshold on E_the / E_kin; 0 means 1e-2 */
    int gravity_bc;      /* amr_gravity_bc of amr_hydro_poisson_root (0: periodic) */
} amr_hydro_params;

typedef struct amr_hydro_ctx amr_hydro_ctx; /* opaque, library-owned */

/* Create a context bound to the current CUDA device and to cuda_stream
 * (a cudaStream_t, NULL for the legacy default stream).  Rejects gamma<=1,
 * cfl<=0, lmax outside 0..7, root_n not a positive multiple of 16,
 * max_patches not a positive multiple of 8, non-periodic boundaries, a
 * limiter, riemann or scheme value outside its enum, minmod_coeff neither 0
 * nor in [1, 2], AMR_SCHEME_VL with lmax > 0 or with AMR_RECON_PPM, a
 * recon value outside its enum, fallback not 0 or 1, dt_min < 0, and
 * dual_energy not 0 or 1, dual_xi < 0, or dual_energy with another scheme,
 * PPM, lmax > 0 or the cell remedies, and a gravity_bc outside its enum. */
amr_status amr_hydro_init(const amr_hydro_params *params, void *cuda_stream,
                          amr_hydro_ctx **out);

/* Free the context's scratch; caller-owned arrays are untouched. */
amr_status amr_hydro_destroy(amr_hydro_ctx *ctx);

/*
 * Register the device arrays of one AMR level (section 2.1).
 *   n_patches       number of patches, a multiple of 8 (whole groups), <= max_patches
 *   U_a, U_b        two FP64 state buffers [n_patches][5][8][8][8]; U_a holds the
 *                   current state on entry, U_b receives the next time level
 *   corner          int32 [n_patches][3]: lower-corner cell index (x,y,z) of each
 *                   patch in level-l cell units
 *   sib             int32 [n_patches][26]: slot of the sibling in direction
 *                   (dx,dy,dz) in {-1,0,1}^3 \ {0}, at index k - (k > 13) with
 *                   k = (dx+1) + 3(dy+1) + 9(dz+1); -1 when that sibling is absent
 *   parent          int32 [n_patches]: parent slot on level l-1 (-1 on level 0)
 *   child_group     int32 [n_patches]: group index on level l+1 of the 8 children,
 *                   -1 for a leaf patch
 * The tables are read once here (device to host) to build the context's
 * neighbour plan; call set_level again after any regrid.  The level's time is
 * set to t.  Errors: AMR_E_INVAL on bad sizes or a table entry out of range,
 * AMR_E_NESTING when a coarse-fine ghost patch has no covering coarse patch.
 */
amr_status amr_hydro_set_level(amr_hydro_ctx *ctx, int level, int n_patches,
                               double *U_a, double *U_b, const int32_t *corner,
                               const int32_t *sib, const int32_t *parent,
                               int32_t *child_group, double t);

/*
 * Levels built by regridding (AMR runs).  bind_level registers caller-owned
 * capacity arrays for level 1..lmax, each sized for max_patches slots
 * (U_a, U_b [max_patches][5][8][8][8] FP64; corner [max_patches][3], sib
 * [max_patches][26], parent, child_group [max_patches] int32, layouts as in
 * amr_hydro_set_level).  The level starts empty; amr_hydro_regrid fills the
 * tables and the state and rewrites them at every regrid.  The child_group
 * array given to amr_hydro_set_level for level 0 is rewritten in the same way.
 */
amr_status amr_hydro_bind_level(amr_hydro_ctx *ctx, int level, double *U_a, double *U_b,
                                int32_t *corner, int32_t *sib, int32_t *parent,
                                int32_t *child_group);

/*
 * Rebuild level+1 from the refinement flags of `level` at its current time
 * (section 2.1): cell criterion and flag buffer (amr_hydro_regrid_flags);
 * a patch gains children only if all 26 sibling positions hold patches
 * (proper nesting); a refined patch keeps its children while any
 * level-(level+1) patch with children has a 26-neighbour position inside it;
 * other unflagged patches lose their children (no explicit derefinement
 * criterion).  Kept children keep their data; new children are interpolated
 * from the parent level (conservative minmod-limited linear interpolation of
 * the conserved variables, with all eight children of a coarse cell falling
 * back to the coarse value when any would have rho<=0 or P<=0).  Existing
 * groups keep their numbers (and their slots' data stays in place) where
 * the new group count allows; the others take the free numbers in
 * increasing order, moved groups (by number) before new ones (by their
 * parents' corners, z, then y, then x), so the numbering depends only on the
 * old and new refined sets.  Synchronises.  AMR_E_NOMEM if the new level
 * exceeds max_patches.
 */
amr_status amr_hydro_regrid(amr_hydro_ctx *ctx, int level);

/*
 * One root-level step of the adaptive time-step W-cycle (section 2.1):
 * level l takes steps dt_l = Eq. (CFL2) until it reaches its parent's time;
 * dt_l grows by up to C_inc to land exactly on the parent's time, or shrinks
 * by up to C_dec to twice the child level's last step; after each step of
 * level l its child level catches up, then flux fix-up + restriction and the
 * regrid of level l+1.  dt0 > 0 fixes the root step, else Eq. (CFL2).
 * cell_updates (may be NULL) receives the number of cell updates of all
 * levels.  Synchronises the host once per level step (for its dt).  With
 * the shared time step on (amr_hydro_set_shared_dt) every level takes one
 * step per root step of the root step's dt: the minimum of Eq. (CFL2) over
 * all levels (section 2.6), no C_dec shrink.
 */
amr_status amr_hydro_advance_root(amr_hydro_ctx *ctx, double dt0, int64_t *cell_updates);

/*
 * Shared (on != 0) or adaptive (0, the default) time-step integration of
 * amr_hydro_advance_root (section 2.6).  AMR_E_INVAL for a NULL context.
 */
amr_status amr_hydro_set_shared_dt(amr_hydro_ctx *ctx, int on);

/* Patch and coarse-fine ghost-patch counts of a level. */
amr_status amr_hydro_level_info(amr_hydro_ctx *ctx, int level, int *n_patches, int *n_ghost);

/* Report which registered buffer holds the level's newest state (0 = U_a,
 * 1 = U_b) and the times of the newest and previous states. */
amr_status amr_hydro_get_state(amr_hydro_ctx *ctx, int level, int *cur_buffer,
                               double *t_cur, double *t_prev);

/* Declare that the caller rewrote the level's newest state buffer (a new
 * initial condition, a restart, an in-place edit): reductions cached from the
 * last step are dropped.  Asynchronous; no device work. */
amr_status amr_hydro_touch_level(amr_hydro_ctx *ctx, int level);

/* Register the dual-energy entropy fields of `level` (params.dual_energy):
 * two FP64 buffers [n_patches][8][8][8] in the slot order of the level's
 * state, S_a holding s = P / rho^(gamma-1) of the current state, S_b
 * receiving the next; they swap with U_a / U_b at every step (the newest
 * is S_a after an even number of steps).  Caller-owned.  For a refined level
 * bound with amr_hydro_bind_level, register buffers of its capacity before
 * the first regrid fills it: S_a pairs with U_a, S_b with U_b.  AMR_E_INVAL
 * for a context without dual energy, a level without patches that is not
 * bound, or equal buffers. */
amr_status amr_hydro_set_entropy(amr_hydro_ctx *ctx, int level, double *S_a, double *S_b);

/*
 * Fill the coarse-fine ghost patches of `level` (>0) at time t by linear
 * interpolation in time between the coarse level's previous and newest
 * states, then conservative minmod-limited linear interpolation in space
 * (section 3.2: ghost zones are filled from siblings, or by interpolation
 * from coarse patches).  advance_level calls this itself; it is exposed for
 * tests.  t must lie in [t_prev, t_cur] of level-1.
 */
amr_status amr_hydro_fill_ghost(amr_hydro_ctx *ctx, int level, double t);

/*
 * Advance every patch group of `level` by one step of size dt with the
 * context's scheme (section 2.2; default MUSCL-Hancock): gather the ghosted
 * tile, reconstruction + limiter, the scheme's predictor, the Riemann solver
 * at every face, conservative update into the other buffer, coarse-fine
 * flux registers, and the CFL reduction of the new state (fused).  dt < 0
 * means: use the device-side dt of the scheme's CFL condition from the
 * latest reduction (no host synchronisation).  If n_unphysical_out is not
 * NULL the call synchronises and stores the number of updated cells with
 * rho<=0 or P<=0 (after the per-cell remedies when params.fallback is set),
 * returning AMR_E_UNPHYSICAL when it is not zero.  With params.dt_min > 0
 * the call synchronises after every attempt and retries the step from the
 * same state with dt x 0.8 while cells stay unphysical, returning
 * AMR_E_UNPHYSICAL once dt < dt_min; the level's time then advances by the
 * dt actually taken.
 */
amr_status amr_hydro_advance_level(amr_hydro_ctx *ctx, int level, double dt,
                                   int64_t *n_unphysical_out);

/*
 * The step of amr_hydro_advance_level for a uniform periodic root grid held on
 * the host (section 3.1 overlaps host-device transfers with the GPU solver
 * through CUDA streams): U_in is copied to the device, advanced one step and
 * the new state copied back into U_out, in z-slabs of 16 cell planes so that
 * the copies in both directions overlap the update.  Results are bitwise
 * those of amr_hydro_advance_level on the same state.
 *   U_in, U_out  host FP64 [5][nz][ny][nx] (the root grid, x fastest); page-
 *                locked memory gives the overlap, pageable memory works but
 *                serialises the copies.  U_out may equal U_in.
 *   dt           > 0: the step size; <= 0: the Eq. (CFL2) dt of U_in, which
 *                needs all of U_in on the device before the first slab steps
 *   dt_next      host double (may be NULL): the Eq. (CFL2) dt of U_out (-1 if
 *                it has no positive signal speed), to pass as the next dt
 * Level 0 must be the whole root grid in the order of
 * amr_hydro_uniform_tables (set with amr_hydro_set_level) and no finer level
 * may hold patches; otherwise AMR_E_INVAL.  The level's device state becomes
 * the new state, as after amr_hydro_advance_level.  The call returns when
 * U_out is complete (it synchronises the context's stream and its two copy
 * streams).  The device keeps two dense staging copies of the grid
 * (2 x 40 bytes per cell), allocated on the first call.
 */
amr_status amr_hydro_advance_host(amr_hydro_ctx *ctx, const double *U_in, double *U_out, double dt,
                                  double *dt_next);

/*
 * Synchronise coarse_level with coarse_level+1 (section 2.2): coarse leaf
 * cells next to a coarse-fine interface get
 * U_c -= (sum dt_f <F_f> - dt_c F_c)/dh_c across their high faces (+= across
 * low faces), then every non-leaf coarse cell becomes the mean of its 8
 * children.  Fine fluxes are summed in a fixed order: bitwise reproducible.
 */
amr_status amr_hydro_flux_fixup(amr_hydro_ctx *ctx, int coarse_level);

/*
 * Time step of Eq. (CFL2) on `level`: C_CFL dh / max over the level's cells
 * of (|vx|+|vy|+|vz|+3 c_s).  dt_out may be a host pointer (the call
 * synchronises) or a device pointer (asynchronous).  Returns AMR_E_UNPHYSICAL
 * (dt_out = -1) if a cell has rho<=0 or P<=0.
 */
amr_status amr_hydro_min_dt(amr_hydro_ctx *ctx, int level, double *dt_out);

/*
 * Refinement flags of `level` (section 2.1): a cell is flagged when its
 * normalised density gradient exceeds theta, i.e.
 * sum_d ((rho_{+d} - rho_{-d})/2)^2 > theta^2 rho^2; a patch is flagged when
 * any of its cells is.  patch_flags_dev: device uint8 [n_patches].
 */
amr_status amr_hydro_regrid_flags(amr_hydro_ctx *ctx, int level, uint8_t *patch_flags_dev);

/* Sum over the level's leaf cells of U dV per variable, FP64, fixed-order
 * tree (deterministic).  out: host double[5].  Synchronises. */
amr_status amr_hydro_conserved_sum(amr_hydro_ctx *ctx, int level, double *out);

/*
 * Where the time of the level path goes (the paper's performance analysis of
 * section 4.1 splits a step the same way).  With timing on, the context
 * records a CUDA event pair around each phase of its level steps on its
 * stream; phases do not nest (a phase inside another counts for the outer
 * one), so together they cover the stream's time between the first and last
 * event, host gaps included:
 *   AMR_PH_GHOST   coarse-fine ghost interpolation (section 3.2)
 *   AMR_PH_STEP    the fused patch-group step and the cell remedies
 *   AMR_PH_FIXUP   flux fix-up and restriction (section 2.2)
 *   AMR_PH_REGRID  refinement flags, the device-side regrid, plans
 *   AMR_PH_DT      time-step reductions read by the host (Eq. CFL2)
 * amr_hydro_phase_times synchronises the stream, returns the milliseconds
 * and calls per phase (host arrays of AMR_N_PHASES) since the last call, and
 * clears them.  Timing off (the default) records nothing.
 */
#define AMR_PH_GHOST 0
#define AMR_PH_STEP 1
#define AMR_PH_FIXUP 2
#define AMR_PH_REGRID 3
#define AMR_PH_DT 4
#define AMR_N_PHASES 5
amr_status amr_hydro_phase_timing(amr_hydro_ctx *ctx, int on);
amr_status amr_hydro_phase_times(amr_hydro_ctx *ctx, double *ms_out, int64_t *calls_out);

/*
 * Independent periodic boxes advanced together (section 4.2 runs many
 * independent periodic domains, one per node; here they share one GPU).
 * set_box registers box `box_id` (< 256): a uniform periodic cube of n^3 cells
 * (n a multiple of 16, edge length 1, so dh = 1/n) with two caller-owned
 * state buffers in the patch layout above (uniform slot order of
 * amr_hydro_uniform_tables).  advance_boxes runs n_steps steps of every listed
 * box with a per-box dt of Eq. (CFL2) evaluated on the device, as one
 * persistent launch per step over all groups of all boxes; the steps are
 * captured once into a CUDA graph and replayed.  dt_log (device, may be NULL)
 * receives [n_steps][n_boxes] FP64 time steps.
 */
amr_status amr_hydro_set_box(amr_hydro_ctx *ctx, int box_id, int n, double *U_a, double *U_b);
amr_status amr_hydro_advance_boxes(amr_hydro_ctx *ctx, int n_boxes, const int *box_ids,
                                   int n_steps, double *dt_log);
amr_status amr_hydro_box_state(amr_hydro_ctx *ctx, int box_id, int *cur_buffer);
/* Dual energy in the box batch (section 2.2 dual-energy formalism, as for a
 * level with amr_hydro_set_entropy): the entropy per unit volume of box
 * box_id, two caller-owned device FP64 buffers [n_patches][8][8][8] in the
 * box's slot order; S_a holds the current field (it pairs with the box's
 * current state buffer).  Every box of an advance_boxes call needs them when
 * params.dual_energy is set (AMR_E_INVAL otherwise, and for a context
 * without dual energy, an unregistered box or equal buffers). */
amr_status amr_hydro_set_box_entropy(amr_hydro_ctx *ctx, int box_id, double *S_a, double *S_b);
/* Launch shape the autotuner picked for the last box set: persistent grid
 * size, contiguous (1) or grid-stride (0) work runs per CTA, interleaved (1)
 * or box-major (0) work order, and its measured time per batch step.
 * Setting the environment variable AMR_HYDRO_AUTOTUNE=0 skips the timing
 * and uses the resident grid, grid-stride, box-major shape. */
amr_status amr_hydro_box_tuning(amr_hydro_ctx *ctx, int *grid, int *chunked, int *interleave,
                                float *ms_per_step);

/*
 * Gravity (section 2.3; Appendix A).  Root level, periodic: the potential of
 * the 7-point discrete Poisson equation
 *   sum_d (phi_{i+e_d} - 2 phi_i + phi_{i-e_d}) / dh^2 = 4 pi G (rho_i - <rho>)
 * by FFT (phi_k = 4 pi G dh^2 rho_k / lambda_k, lambda_k = -2 sum_d
 * (1 - cos(2 pi k_d / N_d)), phi_0 = 0), from the density of level 0's
 * current state (which must hold the whole root grid).  phi: FP64
 * [n_patches][8][8][8] in level 0's slot order; acc: NULL or
 * [n_patches][3][8][8][8] receiving g = -grad phi (x, y, z) by acc_order = 2
 * or 4 point central differences.  Caller-owned, device; asynchronous on
 * the context's stream.  The library's own mixed-radix FFT (twiddle tables
 * and work arrays kept in the context; every root extent's prime factors at
 * most 64, x even).  With
 * params.gravity_bc = AMR_GRAVITY_ISOLATED: the pairwise point-mass
 * potential (no mean subtracted) by zero-padded FFT convolution, the edge
 * cells' differences reading the potential just outside the box.  In the
 * FP32-compute mode the transforms run in FP32 (outputs still FP64).
 */
amr_status amr_hydro_poisson_root(amr_hydro_ctx *ctx, double G, double *phi, double *acc, int acc_order);

/*
 * Refined level (>= 1): every patch solved on its own (8 + 2*5)^3 grid
 * (section 2.3): density from the level's patches, else injected from the
 * parent level's cells; the grid's outermost layer (fixed) and initial guess
 * by quadratic interpolation in space of phi_coarse (the parent level's
 * potential, [n_coarse_patches][8][8][8]; the tensor product of the 1-D
 * quadratic through coarse cells c-1, c, c+1 at the child's offset -1/4 or
 * +1/4, along x, y, z); then `iters` red-black SOR iterations with
 * relaxation factor omega; the active cells' potential into phi
 * ([n_patches][8][8][8]) and, if acc is not NULL, -grad phi into acc
 * ([n_patches][3][8][8][8]) by acc_order = 2 or 4 point central differences.
 * Asynchronous on the context's stream.  FP64, or FP32 in the FP32-compute
 * mode (inputs and outputs FP64).  phi and acc may not overlap each other or
 * phi_coarse (AMR_E_INVAL).
 */
amr_status amr_hydro_poisson_level(amr_hydro_ctx *ctx, int level, double G, double omega, int iters,
                                   const double *phi_coarse, double *phi, double *acc, int acc_order);

/*
 * The same with the parent's potential interpolated linearly in time
 * (section 2.3, adaptive time steps): every parent cell's value is
 * (1 - w) phi_coarse_old + w phi_coarse_new before the spatial
 * interpolation, w = (t - t_old) / (t_new - t_old) of the parent's two
 * potentials (w in [0, 1], else AMR_E_INVAL).
 */
amr_status amr_hydro_poisson_level_t(amr_hydro_ctx *ctx, int level, double G, double omega, int iters,
                                     const double *phi_coarse_old, const double *phi_coarse_new, double w,
                                     double *phi, double *acc, int acc_order);

/*
 * One hydro step of a single-level periodic grid coupled to self-gravity
 * (section 2.3, the operator-unsplit predictor-corrector after Muller &
 * Steinmetz 1995): the MUSCL-Hancock (or CTU) step whose half step also adds
 * (dt/2) (0, rho g, m.g) of each reconstructed face state (CTU: after the
 * normal predictor, before the transverse correction; g = acc_n, the acceleration at
 * t^n, [n_patches][3][8][8][8]); the FFT potential phi_new and acceleration
 * acc_new of the predicted density (as amr_hydro_poisson_root); then
 * m^{n+1} = m* + (dt/2)(rho^n g^n + rho^{n+1} g^{n+1}) and
 * E^{n+1} = E* + (dt/2)(m^n.g^n + m^{n+1}.g^{n+1}).  acc_new is the next
 * step's acc_n; acc_n, phi_new, acc_new and the level's two state buffers
 * must not overlap one another (AMR_E_INVAL).  dt < 0: the device's Eq. (CFL2) dt, and with c_acc > 0 the
 * smaller of it and Eq. (acc), c_acc (dh / max|a|)^(1/2) over acc_n's values
 * (c_acc = 0: Eq. (CFL2) alone; negative or non-finite: AMR_E_INVAL).
 * MUSCL-Hancock or CTU with PLM
 * without dual energy, the remedies or the level retry; AMR_E_INVAL otherwise or with
 * refined levels.  Asynchronous on the context's stream.
 */
amr_status amr_hydro_advance_gravity(amr_hydro_ctx *ctx, double dt, double G, const double *acc_n, double *phi_new,
                                     double *acc_new, int acc_order, double c_acc);

/*
 * Self-gravity inside the adaptive time-step W-cycle of amr_hydro_advance_root
 * (section 2.3 on the section 2.1 hierarchy): after this call every level
 * step is the coupled step -- the predictor with g^n in its half step (g^n
 * of coarse-fine ghost cells interpolated from the coarse level), the
 * potential of the predicted density at the step's end (root: periodic FFT;
 * refined levels: the per-patch 18^3 SOR, iters red-black sweeps at
 * omega, the parent's potential interpolated linearly in time), and the
 * corrector with g^n and g^{n+1}; one Poisson solve per level step, and a
 * level whose patches a regrid changed is solved again at its time.  The
 * call solves every level's potential at its current time.  G >= 0,
 * 0 < omega < 2, iters >= 0, acc_order 2 or 4.  MUSCL-Hancock + PLM on a
 * periodic root, without dual energy, the remedies or the level retry;
 * AMR_E_INVAL otherwise.  The library owns the potentials.
 */
amr_status amr_hydro_set_gravity(amr_hydro_ctx *ctx, double G, double omega, int iters, int acc_order);
/* The newest potential [n_patches][8][8][8] and acceleration
 * [n_patches][3][8][8][8] of `level` copied into caller-owned device arrays
 * (either may be NULL), in the level's slot order.  Synchronises. */
amr_status amr_hydro_level_gravity(amr_hydro_ctx *ctx, int level, double *phi_out, double *acc_out);

/*
 * Discrete adjoint of one uniform periodic MUSCL-Hancock step of size dt (no
 * counterpart in the paper; the reverse of section 2.2's update with dt held
 * fixed): lam_n = (dU^{n+1}/dU^n)^T lam_np1.  U_n, lam_np1, lam_n: device FP64
 * arrays in the level's patch layout.  At kinks the derivative of the branch
 * taken by the forward evaluation is used.
 */
amr_status amr_hydro_step_adjoint(amr_hydro_ctx *ctx, int level, double dt, const double *U_n,
                                  const double *lam_np1, double *lam_n);

const char *amr_hydro_strerror(amr_status s);

/*
 * One step of a uniform periodic grid that allocates no device memory (the
 * paper has no counterpart: it is a calling convention, not a step of the
 * method).  For callers that cannot call cudaMalloc -- applications whose
 * device memory is reserved up front by their own pool allocator, and
 * latency-critical loops that cannot take the device-wide synchronisation
 * cudaMalloc/cudaFree may cause -- since a context allocates its scratch.
 * The step is the one amr_hydro_advance_level runs (same kernel, same
 * results); its scratch (the per-group neighbour table and the reduction
 * scalars) lives in a static device array of AMR_NOALLOC_MAX_GROUPS x 64
 * int32 + 64 bytes (1 MiB) that every GPU loading the library holds until the
 * process exits.
 *   U_old, U_new   device FP64 [n_patches][5][8][8][8] in the slot order of
 *                  amr_hydro_uniform_tables; distinct buffers
 *   nx, ny, nz     cells per dimension, multiples of 16; at most
 *                  AMR_NOALLOC_MAX_GROUPS patch groups (nx ny nz / 4096),
 *                  larger grids are rejected with AMR_E_INVAL and a message
 *   dh, dt         cell width and time step (dt >= 0, from the host)
 *   gamma, cfl     adiabatic index and C_CFL; prec an amr_precision
 *   dt_next_out    device double (may be NULL): Eq. (CFL2) dt of U_new, -1 if
 *                  a cell is unphysical
 *   n_unphysical_out  device uint64 (may be NULL): cells of U_new with
 *                  rho<=0 or P<=0
 * Asynchronous on cuda_stream.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and configures the kernel;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: calls after cudaDeviceReset (or any other
 * teardown of the device's primary context) are not supported.  Every call shares the
 * array and it keeps the last call's contents (each call rebuilds what it
 * reads and zeroes what it accumulates into); calls that overlap on the GPU
 * race on it.
 */
#define AMR_NOALLOC_MAX_GROUPS 4096
amr_status amr_hydro_step_uniform_noalloc(const double *U_old, double *U_new, int nx, int ny, int nz,
                                          double dh, double dt, double gamma, double cfl, int prec,
                                          double *dt_next_out, unsigned long long *n_unphysical_out,
                                          void *cuda_stream);

/* ---- host-side helpers (no device work) ---------------------------------- */

/*
 * Tables of a level fully covered by patches: np[d] patches per dimension
 * (each even), periodic wrap.  Slot order: group g = gx + ngx (gy + ngy gz)
 * with ng = np/2, slot = 8g + px + 2py + 4pz.  Host arrays sized as in
 * amr_hydro_set_level; parent/child_group are filled with -1.
 */
amr_status amr_hydro_uniform_tables(const int np[3], int32_t *corner, int32_t *sib,
                                    int32_t *parent, int32_t *child_group);

/* ---- device-side layout helpers ------------------------------------------ */

/* Dense [5][nz][ny][nx] <-> patch layout of amr_hydro_uniform_tables, on
 * cuda_stream.  n{x,y,z} multiples of 16. */
amr_status amr_hydro_pack_uniform(const double *dense, int nx, int ny, int nz, double *patches,
                                  void *cuda_stream);
amr_status amr_hydro_unpack_uniform(const double *patches, int nx, int ny, int nz, double *dense,
                                    void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* AMR_HYDRO_H */
