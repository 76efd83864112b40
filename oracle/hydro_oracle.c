/*
 * hydro_oracle.c -- plain FP64 CPU oracle for the GAMER-2 patch-group fluid
 * update (Schive et al. 2018, "GAMER-2", section 2.2 Hydrodynamics and
 * section 2.6 Time-step).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * It is written as slow, obviously correct per-cell loops over whole-level
 * dense arrays U[var][z][y][x] (x fastest), never over patch tiles, so that it
 * shares no structure with the CUDA path.  Conserved variables are
 * U = (rho, rho vx, rho vy, rho vz, E); primitives W = (rho, vx, vy, vz, P).
 *
 * Scheme (section 2.2: MUSCL-Hancock "MHM", PLM on primitive variables,
 * van Leer-type limiter, HLLC Riemann solver).  The paper defers the scheme's
 * details to Toro (2009); the readings taken here are:
 *   - slopes on primitives, per component and per dimension,
 *     vL(a,b) = 2ab/(a+b) if ab > 0 else 0 (harmonic van Leer form);
 *   - face states W_{d,-/+} = W -/+ dW_d/2, converted to U;
 *   - Hancock half step: every face state of a cell gets
 *     + (dt/2dh) sum_d [F_d(U_{d,-}) - F_d(U_{d,+})];
 *   - HLLC with Einfeldt/Roe-averaged outer wave speeds, contact speed S*,
 *     Toro's star states, tie rules S_L>=0 -> F_L, S_R<=0 -> F_R,
 *     S*>=0 -> F*_L else F*_R;
 *   - conservative update U^{n+1} = U^n - (dt/dh) sum_d (F_{i+1/2}-F_{i-1/2}).
 * Time step: Eq. (CFL2), dt = C_CFL dh / max(|vx|+|vy|+|vz|+3 c_s).
 *
 * Section 2.2 also lists the other slope limiters and Riemann solvers GAMER
 * offers (generalized minmod, van Albada-type, a hybrid of the generalized
 * minmod and van Leer-type limiters; HLLE after Einfeldt 1991), again
 * deferring their definitions to Toro (2009).  With a = W_i - W_{i-1},
 * b = W_{i+1} - W_i (every limiter gives 0 unless ab > 0):
 *   - generalized minmod, coefficient theta in [1,2]:
 *     sign(a) min(theta|a|, |a+b|/2, theta|b|);
 *   - van Albada-type: ab(a+b)/(a^2+b^2);
 *   - hybrid: sign(a) min(|vL(a,b)|, |generalized minmod(a,b)|);
 *   - HLLE: the HLLC outer speeds S_L, S_R above, F_L if S_L>=0, F_R if
 *     S_R<=0, else (S_R F_L - S_L F_R + S_L S_R (U_R - U_L))/(S_R - S_L).
 *   - Roe: Roe averages, primitive-jump wave strengths and the averaged
 *     Jacobian's right eigenvectors (Toro 2009 ch. 11), Harten-Hyman entropy
 *     fix on the acoustic waves with delta = max(0, lambda~ - lambda(W_L),
 *     lambda(W_R) - lambda~);
 *   - exact: the physical flux of the exact solution at x/t = 0 (the exact
 *     solver below), transverse velocities from the contact's upwind side.
 * or_set_scheme selects them; the default is van Leer-type + HLLC.
 *
 * Scheme (section 2.2 lists the VL variant of MUSCL-Hancock, after Falle 1991
 * and van Leer 2006); reading: a half step with the Riemann fluxes of the
 * cell averages, U* = U^n - (dt/2dh) sum_d [F(U_i, U_i+1) - F(U_i-1, U_i)];
 * the selected limiter's PLM reconstruction of W(U*) to face states
 * W* -/+ (1/2) dW* (no further evolution); the full step with the Riemann fluxes
 * of those face states.  or_set_vl(1) selects it for every later step.
 *
 * Scheme (section 2.2 lists the CTU scheme of Colella 1990 in the variant with
 * six Riemann solves per cell, as in Athena, Stone et al. 2008); reading:
 *   - normal predictor: the face states along d of a cell evolve by d's own
 *     flux difference only, U_{d,-/+} + (dt/2dh) [F_d(U_{d,-}) - F_d(U_{d,+})];
 *   - first fluxes F1 of those states at every face (three solves per cell);
 *   - transverse correction: the face states along d of a cell take
 *     - (dt/2dh) sum_{e != d} [F1_e(i+1/2) - F1_e(i-1/2)] of that cell;
 *   - final fluxes of the corrected states (three more solves) update U^n.
 *   Time step: Eq. (CFL1), dt = C_CFL dh / max(max(|vx|,|vy|,|vz|) + c_s).
 * or_set_ctu(1) selects it for every later step.
 *
 * Reconstruction (section 2.2 lists PPM, Colella & Woodward 1984): face values
 * of a primitive component from the cells i-2..i+2,
 *   W_{i+1/2} = (W_i + W_{i+1})/2 - (dW_{i+1} - dW_i)/6
 * with dW the selected limiter's slope, then the CW84 monotonicity
 * constraints: both faces take W_i at an extremum ((W_R - W_i)(W_i - W_L) <= 0);
 * otherwise with d = W_R - W_L and m = 6 (W_i - (W_L + W_R)/2), d m > d^2 sets
 * W_L = 3 W_i - 2 W_R and d m < -d^2 sets W_R = 3 W_i - 2 W_L.  The face
 * values replace W -/+ dW/2 in every scheme above.  or_set_ppm(1) selects it.
 *
 * Unphysical results (section 2.2 lists GAMER's remedies; or_set_fallback(1)
 * enables the per-cell ones):
 *   (0)   a face whose left or right state has rho <= 0 or P <= 0 has no
 *         flux (NaN), so the cells on both sides count as unphysical;
 *   (i)   the Roe solver checks its two intermediate states U_L + alpha_1 K_1
 *         and U_R - alpha_5 K_5 (and the Roe sound speed); if either has
 *         rho <= 0 or P <= 0 the face takes the HLLE flux instead;
 *   (ii)  a cell whose updated state has rho <= 0 or P <= 0 is recomputed
 *         first order in space and time, unsplit:
 *         U^n - (dt/dh) sum_d [F_d(U_i, U_i+1) - F_d(U_i-1, U_i)] with the
 *         selected solver on cell averages;
 *   (iii) if that is still unphysical, first order dimensionally split: an
 *         x sweep of U^n, a y sweep of its result, a z sweep of that (each
 *         sweep V - (dt/dh)[F(V_i, V_i+1) - F(V_i-1, V_i)] along its axis);
 *   cells still unphysical after (iii) are counted, and the step loop retries
 *   the whole step with dt x 0.8 (iv) down to a minimum dt (v).
 * The fluxes returned for the flux registers stay those of the scheme.
 *
 * Gravity (section 2.3: operator-unsplit predictor-corrector after Muller &
 * Steinmetz 1995); reading: the predictor is the MUSCL-Hancock step whose
 * half step also adds (dt/2) (0, rho g, m.g) of each reconstructed face
 * state, g the cell's acceleration at t^n; the corrector (in oracle/poisson.py)
 * takes g^{n+1} of the predicted density and sets
 * m^{n+1} = m* + (dt/2)(rho^n g^n + rho^{n+1} g^{n+1}), then
 * E^{n+1} = E* + (dt/2)(m^n.g^n + m^{n+1}.g^{n+1}) with the corrected m.
 *
 * Dual energy (section 2.2: the entropy per unit volume s = P / rho^(gamma-1)
 * carried as a passive scalar; or_step_dual, MUSCL-Hancock only).  Reading:
 *   - reconstruction of q = s / rho like a primitive component (the selected
 *     limiter, PLM or PPM), face values s = rho_face q_face, the Hancock
 *     increment (dt/2dh) sum_d [F_s(U_d,-) - F_s(U_d,+)] with F_s = s v_n;
 *   - the scalar flux of a face: the mass flux F_rho times q of its upwind
 *     side (q = s / rho of the left face state if F_rho >= 0, else of the
 *     right one); conservative update of s;
 *   - after the update, with E_kin = |m|^2 / (2 rho) and E_the = E - E_kin:
 *     if E_the < xi E_kin the total energy becomes
 *     E_kin + s rho^(gamma-1) / (gamma-1); otherwise the entropy is reset
 *     from the total energy, s = (gamma-1) E_the / rho^(gamma-1).
 *
 * Every per-cell loop is independent, so the OpenMP static split changes no
 * result: the oracle is bitwise reproducible for any thread count (the
 * paper's section 2.7.1 property).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV 5

static inline int64_t cell_index(int x, int y, int z, int nx, int ny) {
    return ((int64_t)z * ny + y) * nx + x;
}

static inline int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* ---- equation of state (ideal gas) ------------------------------------ */

/* U -> W.  P = (gamma-1)(E - rho|v|^2/2). */
void or_prim(const double *U, double *W, double gamma) {
    double rho = U[0];
    double vx = U[1] / rho, vy = U[2] / rho, vz = U[3] / rho;
    double ekin = 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    W[0] = rho;
    W[1] = vx;
    W[2] = vy;
    W[3] = vz;
    W[4] = (gamma - 1.0) * (U[4] - ekin);
}

/* W -> U.  E = P/(gamma-1) + rho|v|^2/2. */
void or_cons(const double *W, double *U, double gamma) {
    double rho = W[0];
    U[0] = rho;
    U[1] = rho * W[1];
    U[2] = rho * W[2];
    U[3] = rho * W[3];
    U[4] = W[4] / (gamma - 1.0) + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

/* Physical Euler flux along direction d (0=x,1=y,2=z) of conserved state U. */
void or_flux(const double *U, int d, double gamma, double *F) {
    double W[NV];
    or_prim(U, W, gamma);
    double vn = W[1 + d], P = W[4];
    F[0] = U[0] * vn;
    F[1] = U[1] * vn;
    F[2] = U[2] * vn;
    F[3] = U[3] * vn;
    F[1 + d] += P;
    F[4] = (U[4] + P) * vn;
}

/* Sound speed c_s = sqrt(gamma P / rho). */
static double sound_speed(const double *W, double gamma) {
    return sqrt(gamma * W[4] / W[0]);
}

/* van Leer-type slope limiter (section 2.2), harmonic form. */
double or_vanleer(double a, double b) {
    double ab = a * b;
    return ab > 0.0 ? 2.0 * ab / (a + b) : 0.0;
}

/* ---- scheme selection (section 2.2: limiters and Riemann solvers) ------- */

/* limiter: 0 van Leer-type, 1 generalized minmod, 2 van Albada-type,
 * 3 hybrid generalized minmod / van Leer-type; riemann: 0 HLLC, 1 HLLE;
 * theta: the generalized minmod coefficient. */
static int or_limiter_id = 0, or_riemann_id = 0, or_vl = 0, or_ctu = 0, or_ppm = 0, or_fallback = 0;
/* gravity predictor: the cell-centred acceleration g^n [3][cell] of the
 * step in progress (or_step_gravity_predictor) */
static const double *or_grav_g = NULL;

/* Gravity in the half step of cell i: + (dt/2) (0, rho g, m.g) of each of
 * its six reconstructed face states Uf, added to the predicted states FS
 * (MUSCL-Hancock after the Hancock increment; CTU after the normal
 * predictor, before the transverse correction). */
static void or_grav_faces(double *FS, double Uf[6][NV], const double *gfield, int64_t i, int64_t n, double dt) {
    double g[3];
    for (int d = 0; d < 3; d++) g[d] = gfield[(int64_t)d * n + i];
    for (int f = 0; f < 6; f++) {
        for (int d = 0; d < 3; d++) FS[((int64_t)f * NV + 1 + d) * n + i] += 0.5 * dt * (Uf[f][0] * g[d]);
        FS[((int64_t)f * NV + 4) * n + i] += 0.5 * dt * (Uf[f][1] * g[0] + Uf[f][2] * g[1] + Uf[f][3] * g[2]);
    }
}
/* dual energy: the entropy fields of the step in progress (or_step_dual) */
static const double *or_de_S = NULL;
static double *or_de_Snew = NULL, or_de_xi = 0.0;
static double *or_de_FXs_out = NULL; /* the scalar's face fluxes [3][cells] (or_step_dual_fx) */
static double or_theta = 1.5;

void or_set_vl(int on) { or_vl = on; }
void or_set_ctu(int on) { or_ctu = on; }
void or_set_ppm(int on) { or_ppm = on; }
void or_set_fallback(int on) { or_fallback = on; }

/* Cells the per-cell remedies handled since the last reset: fixed by (ii),
 * fixed by (iii), still unphysical (test instrumentation). */
static int64_t or_fb_count[3];
void or_fallback_counts(int64_t *out, int reset) {
    for (int k = 0; k < 3; k++) {
        out[k] = or_fb_count[k];
        if (reset) or_fb_count[k] = 0;
    }
}

void or_set_scheme(int limiter, int riemann, double theta) {
    or_limiter_id = limiter;
    or_riemann_id = riemann;
    or_theta = theta;
}

/* generalized minmod: sign(a) min(theta|a|, |a+b|/2, theta|b|) if ab > 0 */
double or_gminmod(double a, double b, double theta) {
    if (!(a * b > 0.0)) return 0.0;
    double m = theta * fabs(a);
    double t = theta * fabs(b);
    if (t < m) m = t;
    t = 0.5 * fabs(a + b);
    if (t < m) m = t;
    return a > 0.0 ? m : -m;
}

/* van Albada-type: ab(a+b)/(a^2+b^2) if ab > 0 */
double or_albada(double a, double b) {
    double ab = a * b;
    return ab > 0.0 ? ab * (a + b) / (a * a + b * b) : 0.0;
}

/* hybrid: the smaller in magnitude of the van Leer-type and generalized
 * minmod slopes (both carry the sign of a when ab > 0) */
double or_vl_gminmod(double a, double b, double theta) {
    if (!(a * b > 0.0)) return 0.0;
    double v = fabs(or_vanleer(a, b)), m = fabs(or_gminmod(a, b, theta));
    if (v < m) m = v;
    return a > 0.0 ? m : -m;
}

/* the selected limiter */
double or_slope(double a, double b) {
    switch (or_limiter_id) {
        case 1: return or_gminmod(a, b, or_theta);
        case 2: return or_albada(a, b);
        case 3: return or_vl_gminmod(a, b, or_theta);
        default: return or_vanleer(a, b);
    }
}

/* PPM face values (W_L at i-1/2, W_R at i+1/2) of cell i from w[0..4] =
 * W_{i-2..i+2} of one primitive component (Colella & Woodward 1984,
 * interpolation with the selected limiter's slopes, then monotonicity). */
void or_ppm_faces(const double *w, double *wl, double *wr) {
    double dm = or_slope(w[1] - w[0], w[2] - w[1]);
    double d0 = or_slope(w[2] - w[1], w[3] - w[2]);
    double dp = or_slope(w[3] - w[2], w[4] - w[3]);
    double l = 0.5 * (w[1] + w[2]) - (d0 - dm) / 6.0;
    double r = 0.5 * (w[2] + w[3]) - (dp - d0) / 6.0;
    double c = w[2];
    if ((r - c) * (c - l) <= 0.0) {
        l = c;
        r = c;
    } else {
        double d = r - l, m = 6.0 * (c - 0.5 * (l + r));
        if (d * m > d * d)
            l = 3.0 * c - 2.0 * r;
        else if (d * m < -d * d)
            r = 3.0 * c - 2.0 * l;
    }
    *wl = l;
    *wr = r;
}

/* With the remedies on, every solver gives a face whose left or right state
 * has rho <= 0 or P <= 0 no flux (every component NaN), so the cells on both
 * sides of it count as unphysical and take the cell remedies.  Compares only. */
static int or_no_flux(const double *WL, const double *WR, double *F) {
    if (!or_fallback || (WL[0] > 0.0 && WL[4] > 0.0 && WR[0] > 0.0 && WR[4] > 0.0)) return 0;
    for (int v = 0; v < NV; v++) F[v] = NAN;
    return 1;
}

/* ---- HLLC Riemann solver (section 2.2; Toro 2009 ch. 10 form) ---------- */

/* Flux across a face normal to direction d, left state UL, right state UR. */
void or_hllc(const double *UL, const double *UR, int d, double gamma, double *F) {
    double WL[NV], WR[NV], FL[NV], FR[NV];
    or_prim(UL, WL, gamma);
    or_prim(UR, WR, gamma);
    if (or_no_flux(WL, WR, F)) return;
    or_flux(UL, d, gamma, FL);
    or_flux(UR, d, gamma, FR);

    double rl = WL[0], pl = WL[4], ul = WL[1 + d];
    double rr = WR[0], pr = WR[4], ur = WR[1 + d];
    double cl = sound_speed(WL, gamma), cr = sound_speed(WR, gamma);

    /* Roe averages (Einfeldt/Batten outer speed estimate). */
    double sl = sqrt(rl), sr = sqrt(rr);
    double vt[3];
    for (int k = 0; k < 3; k++) vt[k] = (sl * WL[1 + k] + sr * WR[1 + k]) / (sl + sr);
    double hl = (UL[4] + pl) / rl, hr = (UR[4] + pr) / rr;
    double ht = (sl * hl + sr * hr) / (sl + sr);
    double ct = sqrt((gamma - 1.0) * (ht - 0.5 * (vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2])));

    double a = ul - cl, b = vt[d] - ct;
    double SL = (a <= b) ? a : b;
    a = ur + cr;
    b = vt[d] + ct;
    double SR = (a >= b) ? a : b;

    if (SL >= 0.0) {
        for (int v = 0; v < NV; v++) F[v] = FL[v];
        return;
    }
    if (SR <= 0.0) {
        for (int v = 0; v < NV; v++) F[v] = FR[v];
        return;
    }
    double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
                (rl * (SL - ul) - rr * (SR - ur));
    /* side K = L if S* >= 0 else R */
    const double *UK = (Ss >= 0.0) ? UL : UR;
    const double *WK = (Ss >= 0.0) ? WL : WR;
    const double *FK = (Ss >= 0.0) ? FL : FR;
    double SK = (Ss >= 0.0) ? SL : SR;
    double rK = WK[0], uK = WK[1 + d], pK = WK[4];
    double fac = rK * (SK - uK) / (SK - Ss);
    double Us[NV];
    Us[0] = fac;
    for (int k = 0; k < 3; k++) Us[1 + k] = fac * WK[1 + k];
    Us[1 + d] = fac * Ss;
    Us[4] = fac * (UK[4] / rK + (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
    for (int v = 0; v < NV; v++) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

int or_exact_star(double rl, double ul, double pl, double rr, double ur, double pr,
                  double gamma, double *pstar, double *ustar);
void or_exact_sample(double rl, double ul, double pl, double rr, double ur, double pr,
                     double gamma, const double *xi, int n, double *rho, double *u,
                     double *p);

/* ---- HLLE Riemann solver (section 2.2; Einfeldt 1991) ------------------ */

/* Flux across a face normal to d with the HLLC solver's outer wave speeds. */
void or_hlle(const double *UL, const double *UR, int d, double gamma, double *F) {
    double WL[NV], WR[NV], FL[NV], FR[NV];
    or_prim(UL, WL, gamma);
    or_prim(UR, WR, gamma);
    if (or_no_flux(WL, WR, F)) return;
    or_flux(UL, d, gamma, FL);
    or_flux(UR, d, gamma, FR);
    double rl = WL[0], pl = WL[4], ul = WL[1 + d];
    double rr = WR[0], pr = WR[4], ur = WR[1 + d];
    double cl = sound_speed(WL, gamma), cr = sound_speed(WR, gamma);
    double sl = sqrt(rl), sr = sqrt(rr);
    double vt[3];
    for (int k = 0; k < 3; k++) vt[k] = (sl * WL[1 + k] + sr * WR[1 + k]) / (sl + sr);
    double hl = (UL[4] + pl) / rl, hr = (UR[4] + pr) / rr;
    double ht = (sl * hl + sr * hr) / (sl + sr);
    double ct = sqrt((gamma - 1.0) * (ht - 0.5 * (vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2])));
    double a = ul - cl, b = vt[d] - ct;
    double SL = (a <= b) ? a : b;
    a = ur + cr;
    b = vt[d] + ct;
    double SR = (a >= b) ? a : b;
    if (SL >= 0.0) {
        for (int v = 0; v < NV; v++) F[v] = FL[v];
        return;
    }
    if (SR <= 0.0) {
        for (int v = 0; v < NV; v++) F[v] = FR[v];
        return;
    }
    for (int v = 0; v < NV; v++) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
}

/* ---- Roe's solver (section 2.2; Roe 1981, Toro 2009 ch. 11) ------------- */

/* F = (F_L + F_R)/2 - (1/2) sum_k |lambda_k| alpha_k K_k with Roe averages,
 * wave strengths of the primitive jumps and right eigenvectors of the
 * averaged Jacobian; Harten-Hyman entropy fix on the two acoustic waves:
 * delta = max(0, lambda~ - lambda(W_L), lambda(W_R) - lambda~), and
 * |lambda~| < delta becomes (lambda~^2 + delta^2)/(2 delta). */
void or_roe(const double *UL, const double *UR, int d, double gamma, double *F) {
    double WL[NV], WR[NV], FL[NV], FR[NV];
    or_prim(UL, WL, gamma);
    or_prim(UR, WR, gamma);
    if (or_no_flux(WL, WR, F)) return;
    or_flux(UL, d, gamma, FL);
    or_flux(UR, d, gamma, FR);
    double sl = sqrt(WL[0]), sr = sqrt(WR[0]);
    double u[3];
    for (int k = 0; k < 3; k++) u[k] = (sl * WL[1 + k] + sr * WR[1 + k]) / (sl + sr);
    double hl = (UL[4] + WL[4]) / WL[0], hr = (UR[4] + WR[4]) / WR[0];
    double H = (sl * hl + sr * hr) / (sl + sr);
    double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double a = sqrt((gamma - 1.0) * (H - 0.5 * q2));
    double r = sl * sr; /* Roe-averaged density */
    double un = u[d];
    double drho = WR[0] - WL[0], dp = WR[4] - WL[4], dun = WR[1 + d] - WL[1 + d];
    double a1 = (dp - r * a * dun) / (2.0 * a * a);
    double a2 = drho - dp / (a * a);
    double a5 = (dp + r * a * dun) / (2.0 * a * a);
    double l1 = fabs(un - a), l2 = fabs(un), l5 = fabs(un + a);
    double cl = sound_speed(WL, gamma), cr = sound_speed(WR, gamma);
    double del = 0.0, t;
    t = (un - a) - (WL[1 + d] - cl);
    if (t > del) del = t;
    t = (WR[1 + d] - cr) - (un - a);
    if (t > del) del = t;
    if (l1 < del) l1 = (l1 * l1 + del * del) / (2.0 * del);
    del = 0.0;
    t = (un + a) - (WL[1 + d] + cl);
    if (t > del) del = t;
    t = (WR[1 + d] + cr) - (un + a);
    if (t > del) del = t;
    if (l5 < del) l5 = (l5 * l5 + del * del) / (2.0 * del);
    /* D = sum_k |lambda_k| alpha_k K_k:
     * K_1,5 = (1, u -/+ a n, H -/+ un a), K_2 = (1, u, q2/2),
     * shear: rho~ dv_t (0, e_t, u_t) for each transverse direction t */
    double D[NV];
    D[0] = l1 * a1 + l2 * a2 + l5 * a5;
    for (int k = 0; k < 3; k++) D[1 + k] = (l1 * a1 + l2 * a2 + l5 * a5) * u[k];
    D[1 + d] += (l5 * a5 - l1 * a1) * a;
    D[4] = l1 * a1 * (H - un * a) + l2 * a2 * 0.5 * q2 + l5 * a5 * (H + un * a);
    for (int k = 0; k < 3; k++) {
        if (k == d) continue;
        double sh = l2 * r * (WR[1 + k] - WL[1 + k]);
        D[1 + k] += sh;
        D[4] += sh * u[k];
    }
    for (int v = 0; v < NV; v++) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * D[v];
    if (or_fallback) {
        /* (i): the intermediate states U_L + a1 K1 and U_R - a5 K5 */
        double Us[2][NV];
        for (int s2 = 0; s2 < 2; s2++) {
            const double al = s2 == 0 ? a1 : -a5, sg = s2 == 0 ? -1.0 : 1.0;
            const double *U0 = s2 == 0 ? UL : UR;
            Us[s2][0] = U0[0] + al;
            for (int k = 0; k < 3; k++) Us[s2][1 + k] = U0[1 + k] + al * u[k];
            Us[s2][1 + d] += al * sg * a;
            Us[s2][4] = U0[4] + al * (H + sg * un * a);
        }
        int bad = !(a > 0.0);
        for (int s2 = 0; s2 < 2 && !bad; s2++) {
            double Wt[NV];
            or_prim(Us[s2], Wt, gamma);
            bad = !(Wt[0] > 0.0) || !(Wt[4] > 0.0);
        }
        if (bad) or_hlle(UL, UR, d, gamma, F);
    }
}

/* ---- exact Riemann solver flux (section 2.2; Toro 2009 ch. 4) ----------- */

/* Godunov flux: the physical flux of the exact solution at x/t = 0 (the
 * normal velocity, density and pressure from or_exact_sample; the
 * transverse velocities of the side of the contact x/t = 0 lies on,
 * the left one when the contact does not move). */
void or_exact_flux(const double *UL, const double *UR, int d, double gamma, double *F) {
    double WL[NV], WR[NV], W[NV], U[NV];
    or_prim(UL, WL, gamma);
    or_prim(UR, WR, gamma);
    if (or_no_flux(WL, WR, F)) return;
    double ps, us, xi = 0.0, r, v, q;
    or_exact_star(WL[0], WL[1 + d], WL[4], WR[0], WR[1 + d], WR[4], gamma, &ps, &us);
    or_exact_sample(WL[0], WL[1 + d], WL[4], WR[0], WR[1 + d], WR[4], gamma, &xi, 1, &r, &v, &q);
    const double *Wt = (us >= 0.0) ? WL : WR;
    W[0] = r;
    for (int k = 0; k < 3; k++) W[1 + k] = Wt[1 + k];
    W[1 + d] = v;
    W[4] = q;
    or_cons(W, U, gamma);
    or_flux(U, d, gamma, F);
}

/* the selected Riemann solver: 0 HLLC, 1 HLLE, 2 Roe, 3 exact */
void or_riemann(const double *UL, const double *UR, int d, double gamma, double *F) {
    if (or_riemann_id == 1)
        or_hlle(UL, UR, d, gamma, F);
    else if (or_riemann_id == 2)
        or_roe(UL, UR, d, gamma, F);
    else if (or_riemann_id == 3)
        or_exact_flux(UL, UR, d, gamma, F);
    else
        or_hllc(UL, UR, d, gamma, F);
}

/* ---- time step, Eq. (CFL2) --------------------------------------------- */

/* max over cells of |vx|+|vy|+|vz|+3 c_s.  Returns -1 if a cell has
 * rho<=0 or P<=0 (unphysical: no floors in the oracle). */
double or_max_speed(const double *U, int64_t ncell, double gamma) {
    double smax = 0.0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(max : smax) reduction(| : bad)
    for (int64_t i = 0; i < ncell; i++) {
        double u[NV], W[NV];
        for (int v = 0; v < NV; v++) u[v] = U[v * ncell + i];
        or_prim(u, W, gamma);
        if (!(W[0] > 0.0) || !(W[4] > 0.0)) {
            bad = 1;
            continue;
        }
        double s = fabs(W[1]) + fabs(W[2]) + fabs(W[3]) + 3.0 * sound_speed(W, gamma);
        if (s > smax) smax = s;
    }
    return bad ? -1.0 : smax;
}

/* Eq. (CFL1): max over cells of max(|vx|,|vy|,|vz|) + c_s; -1 if a cell is
 * unphysical. */
double or_max_speed1(const double *U, int64_t ncell, double gamma) {
    double smax = 0.0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(max : smax) reduction(| : bad)
    for (int64_t i = 0; i < ncell; i++) {
        double u[NV], W[NV];
        for (int v = 0; v < NV; v++) u[v] = U[v * ncell + i];
        or_prim(u, W, gamma);
        if (!(W[0] > 0.0) || !(W[4] > 0.0)) {
            bad = 1;
            continue;
        }
        double m = fabs(W[1]);
        if (fabs(W[2]) > m) m = fabs(W[2]);
        if (fabs(W[3]) > m) m = fabs(W[3]);
        double s = m + sound_speed(W, gamma);
        if (s > smax) smax = s;
    }
    return bad ? -1.0 : smax;
}

double or_dt_cfl1(const double *U, int64_t ncell, double gamma, double cfl, double dh) {
    double s = or_max_speed1(U, ncell, gamma);
    if (s <= 0.0) return -1.0;
    return cfl * dh / s;
}

double or_dt_cfl2(const double *U, int64_t ncell, double gamma, double cfl, double dh) {
    double s = or_max_speed(U, ncell, gamma);
    if (s <= 0.0) return -1.0;
    return cfl * dh / s;
}

/* ---- one MUSCL-Hancock step on a uniform periodic grid ----------------- */

/*
 * U, Unew: [5][nz][ny][nx] FP64.  dh: cell width, dt: time step.
 * Returns the number of cells of Unew with rho<=0 or P<=0.
 */
int64_t or_step_periodic_fx(const double *U, double *Unew, int nx, int ny, int nz,
                            double dh, double dt, double gamma, double *FX_out);

int64_t or_step_periodic(const double *U, double *Unew, int nx, int ny, int nz,
                         double dh, double dt, double gamma) {
    return or_step_periodic_fx(U, Unew, nx, ny, nz, dh, dt, gamma, NULL);
}

/* Whether a conserved state has rho > 0 and P > 0. */
static int or_physical(const double *u, double gamma) {
    double w[NV];
    or_prim(u, w, gamma);
    return w[0] > 0.0 && w[4] > 0.0;
}

/* The first-order update of one cell along d from V_m, V_0, V_p (cells i-1,
 * i, i+1 along d): V_0 - r [F(V_0, V_p) - F(V_m, V_0)]. */
static void or_sweep(const double *Vm, const double *V0, const double *Vp, int d, double r, double gamma,
                     double *out) {
    double Fp[NV], Fm[NV];
    or_riemann(V0, Vp, d, gamma, Fp);
    or_riemann(Vm, V0, d, gamma, Fm);
    for (int v = 0; v < NV; v++) out[v] = V0[v] - r * (Fp[v] - Fm[v]);
}

/* Remedies (ii) and (iii) for cell (x, y, z) of U^n: the first-order unsplit
 * update, and if that is unphysical the first-order split one (x, then y,
 * then z sweeps over the cell's 3x3x3 neighbourhood).  Writes the state to
 * out and returns whether it is physical. */
static int or_fallback_cell(const double *U, int nx, int ny, int nz, int x, int y, int z, double dh, double dt,
                            double gamma, double *out) {
    const int64_t n = (int64_t)nx * ny * nz;
    double B[3][3][3][NV]; /* B[k][j][i] = U^n at (x+i-1, y+j-1, z+k-1) */
    for (int k = 0; k < 3; k++)
        for (int j = 0; j < 3; j++)
            for (int i = 0; i < 3; i++) {
                int64_t c = cell_index(wrap(x + i - 1, nx), wrap(y + j - 1, ny), wrap(z + k - 1, nz), nx, ny);
                for (int v = 0; v < NV; v++) B[k][j][i][v] = U[v * n + c];
            }
    const double r = dt / dh;
    /* (ii) */
    double div[NV] = {0, 0, 0, 0, 0};
    for (int d = 0; d < 3; d++) {
        const double *um = d == 0 ? B[1][1][0] : (d == 1 ? B[1][0][1] : B[0][1][1]);
        const double *up = d == 0 ? B[1][1][2] : (d == 1 ? B[1][2][1] : B[2][1][1]);
        double Fp[NV], Fm[NV];
        or_riemann(B[1][1][1], up, d, gamma, Fp);
        or_riemann(um, B[1][1][1], d, gamma, Fm);
        for (int v = 0; v < NV; v++) div[v] += Fp[v] - Fm[v];
    }
    for (int v = 0; v < NV; v++) out[v] = B[1][1][1][v] - r * div[v];
    if (or_physical(out, gamma)) {
#pragma omp atomic
        or_fb_count[0]++;
        return 1;
    }
    /* (iii) */
    double X[3][3][NV], Y[3][NV];
    for (int k = 0; k < 3; k++)
        for (int j = 0; j < 3; j++) or_sweep(B[k][j][0], B[k][j][1], B[k][j][2], 0, r, gamma, X[k][j]);
    for (int k = 0; k < 3; k++) or_sweep(X[k][0], X[k][1], X[k][2], 1, r, gamma, Y[k]);
    or_sweep(Y[0], Y[1], Y[2], 2, r, gamma, out);
    const int ok = or_physical(out, gamma);
#pragma omp atomic
    or_fb_count[ok ? 1 : 2]++;
    return ok;
}

/* Riemann fluxes FX[d][var][cell] through the high face of every cell along d
 * from the face states FS[face][var][cell] (face 2d+1 of cell i against face
 * 2d of cell i+1). */
static void or_face_fluxes(const double *FS, double *FX, int nx, int ny, int nz, double gamma) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int dims[3] = {nx, ny, nz};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int c[3] = {x, y, z};
                int64_t i = cell_index(x, y, z, nx, ny);
                for (int d = 0; d < 3; d++) {
                    int cp[3] = {c[0], c[1], c[2]};
                    cp[d] = wrap(c[d] + 1, dims[d]);
                    int64_t ip = cell_index(cp[0], cp[1], cp[2], nx, ny);
                    double UL[NV], UR[NV], F[NV];
                    for (int v = 0; v < NV; v++) {
                        UL[v] = FS[((int64_t)(2 * d + 1) * NV + v) * n + i];
                        UR[v] = FS[((int64_t)(2 * d) * NV + v) * n + ip];
                    }
                    or_riemann(UL, UR, d, gamma, F);
                    for (int v = 0; v < NV; v++) FX[((int64_t)d * NV + v) * n + i] = F[v];
                }
            }
}

/* Same step; if FX_out is not NULL it receives the interface fluxes
 * FX_out[d][var][cell] through the high face (i+1/2 along d) of every cell. */
int64_t or_step_periodic_fx(const double *U, double *Unew, int nx, int ny, int nz,
                            double dh, double dt, double gamma, double *FX_out) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int dims[3] = {nx, ny, nz};
    double *W = (double *)malloc(sizeof(double) * NV * n);
    /* face states after the Hancock half step: FS[face][var][cell],
     * face = 2*d + s, s=0 the low (-) face, s=1 the high (+) face */
    double *FS = (double *)malloc(sizeof(double) * 6 * NV * n);
    /* interface fluxes: FX[d][var][cell] is the flux through the high face
     * of the cell along d (i.e. at i+1/2) */
    double *FX = (double *)malloc(sizeof(double) * 3 * NV * n);

    /* 1. primitives (VL: of the half-step state U* from the Riemann fluxes
     *    of the cell averages) */
    double *Uh = NULL;
    if (or_vl) {
        Uh = (double *)malloc(sizeof(double) * NV * n);
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    int c[3] = {x, y, z};
                    int64_t i = cell_index(x, y, z, nx, ny);
                    double ui[NV], div[NV] = {0, 0, 0, 0, 0};
                    for (int v = 0; v < NV; v++) ui[v] = U[v * n + i];
                    for (int d = 0; d < 3; d++) {
                        int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
                        cm[d] = wrap(c[d] - 1, dims[d]);
                        cp[d] = wrap(c[d] + 1, dims[d]);
                        int64_t im = cell_index(cm[0], cm[1], cm[2], nx, ny);
                        int64_t ip = cell_index(cp[0], cp[1], cp[2], nx, ny);
                        double um[NV], up[NV], Fm[NV], Fp[NV];
                        for (int v = 0; v < NV; v++) {
                            um[v] = U[v * n + im];
                            up[v] = U[v * n + ip];
                        }
                        or_riemann(um, ui, d, gamma, Fm);
                        or_riemann(ui, up, d, gamma, Fp);
                        for (int v = 0; v < NV; v++) div[v] += Fp[v] - Fm[v];
                    }
                    for (int v = 0; v < NV; v++) Uh[v * n + i] = ui[v] - 0.5 * dt / dh * div[v];
                }
    }
    const double *Ur = or_vl ? Uh : U;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double u[NV], w[NV];
        for (int v = 0; v < NV; v++) u[v] = Ur[v * n + i];
        or_prim(u, w, gamma);
        for (int v = 0; v < NV; v++) W[v * n + i] = w[v];
    }
    /* dual energy: q = s / rho, the scalar's face values after the Hancock
     * step and its face fluxes */
    double *Q = NULL, *FSs = NULL, *FXs = NULL;
    if (or_de_S) {
        Q = (double *)malloc(sizeof(double) * n);
        FSs = (double *)malloc(sizeof(double) * 6 * n);
        FXs = (double *)malloc(sizeof(double) * 3 * n);
        for (int64_t i = 0; i < n; i++) Q[i] = or_de_S[i] / W[i];
    }

    /* 2.-3. limited slopes, face states, Hancock half step */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int c[3] = {x, y, z};
                int64_t i = cell_index(x, y, z, nx, ny);
                double w[NV], Wf[6][NV], Uf[6][NV];
                for (int v = 0; v < NV; v++) w[v] = W[v * n + i];
                for (int d = 0; d < 3; d++) {
                    int64_t is[5]; /* cells i-2 .. i+2 along d */
                    for (int k = 0; k < 5; k++) {
                        int ck[3] = {c[0], c[1], c[2]};
                        ck[d] = wrap(c[d] + k - 2, dims[d]);
                        is[k] = cell_index(ck[0], ck[1], ck[2], nx, ny);
                    }
                    for (int v = 0; v < NV; v++) {
                        if (or_ppm) {
                            double w5[5];
                            for (int k = 0; k < 5; k++) w5[k] = W[v * n + is[k]];
                            or_ppm_faces(w5, &Wf[2 * d][v], &Wf[2 * d + 1][v]);
                        } else {
                            double slope = or_slope(w[v] - W[v * n + is[1]], W[v * n + is[3]] - w[v]);
                            Wf[2 * d][v] = w[v] - 0.5 * slope;
                            Wf[2 * d + 1][v] = w[v] + 0.5 * slope;
                        }
                    }
                }
                for (int f = 0; f < 6; f++) or_cons(Wf[f], Uf[f], gamma);
                if (or_vl) { /* the face states are already at the half step */
                    for (int f = 0; f < 6; f++)
                        for (int v = 0; v < NV; v++) FS[((int64_t)f * NV + v) * n + i] = Uf[f][v];
                    continue;
                }
                if (or_ctu) { /* CTU normal predictor: each direction's own flux difference */
                    for (int d = 0; d < 3; d++) {
                        double Fm[NV], Fp[NV];
                        or_flux(Uf[2 * d], d, gamma, Fm);
                        or_flux(Uf[2 * d + 1], d, gamma, Fp);
                        for (int s2 = 0; s2 < 2; s2++)
                            for (int v = 0; v < NV; v++)
                                FS[((int64_t)(2 * d + s2) * NV + v) * n + i] =
                                    Uf[2 * d + s2][v] + 0.5 * dt / dh * (Fm[v] - Fp[v]);
                    }
                    if (or_grav_g) or_grav_faces(FS, Uf, or_grav_g, i, n, dt);
                    continue;
                }
                double inc[NV] = {0, 0, 0, 0, 0};
                for (int d = 0; d < 3; d++) {
                    double Fm[NV], Fp[NV];
                    or_flux(Uf[2 * d], d, gamma, Fm);
                    or_flux(Uf[2 * d + 1], d, gamma, Fp);
                    for (int v = 0; v < NV; v++) inc[v] += Fm[v] - Fp[v];
                }
                for (int f = 0; f < 6; f++)
                    for (int v = 0; v < NV; v++)
                        FS[((int64_t)f * NV + v) * n + i] = Uf[f][v] + 0.5 * dt / dh * inc[v];
                if (or_grav_g) or_grav_faces(FS, Uf, or_grav_g, i, n, dt);
                if (or_de_S) { /* the entropy scalar: face values s = rho_f q_f, Hancock step */
                    double sf[6], incs = 0.0;
                    for (int d = 0; d < 3; d++) {
                        double qm, qp;
                        int64_t is[5];
                        for (int k = 0; k < 5; k++) {
                            int ck[3] = {c[0], c[1], c[2]};
                            ck[d] = wrap(c[d] + k - 2, dims[d]);
                            is[k] = cell_index(ck[0], ck[1], ck[2], nx, ny);
                        }
                        if (or_ppm) {
                            double q5[5];
                            for (int k = 0; k < 5; k++) q5[k] = Q[is[k]];
                            or_ppm_faces(q5, &qm, &qp);
                        } else {
                            double slope = or_slope(Q[i] - Q[is[1]], Q[is[3]] - Q[i]);
                            qm = Q[i] - 0.5 * slope;
                            qp = Q[i] + 0.5 * slope;
                        }
                        sf[2 * d] = Wf[2 * d][0] * qm;
                        sf[2 * d + 1] = Wf[2 * d + 1][0] * qp;
                        incs += sf[2 * d] * Wf[2 * d][1 + d] - sf[2 * d + 1] * Wf[2 * d + 1][1 + d];
                    }
                    for (int f = 0; f < 6; f++) FSs[(int64_t)f * n + i] = sf[f] + 0.5 * dt / dh * incs;
                }
            }

    /* 4. Riemann solver at every face i+1/2: left = high face state of cell i,
     *    right = low face state of cell i+1 */
    or_face_fluxes(FS, FX, nx, ny, nz, gamma);
    if (or_de_S) { /* scalar flux: mass flux times q of the upwind face state */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    int c[3] = {x, y, z};
                    int64_t i = cell_index(x, y, z, nx, ny);
                    for (int d = 0; d < 3; d++) {
                        int cp[3] = {c[0], c[1], c[2]};
                        cp[d] = wrap(c[d] + 1, dims[d]);
                        int64_t ip = cell_index(cp[0], cp[1], cp[2], nx, ny);
                        double fr = FX[((int64_t)d * NV + 0) * n + i];
                        double q = fr >= 0.0 ? FSs[(int64_t)(2 * d + 1) * n + i] / FS[((int64_t)(2 * d + 1) * NV) * n + i]
                                             : FSs[(int64_t)(2 * d) * n + ip] / FS[((int64_t)(2 * d) * NV) * n + ip];
                        FXs[(int64_t)d * n + i] = fr * q;
                    }
                }
    }
    if (or_ctu) {
        /* CTU: transverse correction of the face states by the first fluxes,
         * then the final fluxes */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    int c[3] = {x, y, z};
                    int64_t i = cell_index(x, y, z, nx, ny);
                    double div[3][NV]; /* F1_e(i+1/2) - F1_e(i-1/2) of this cell along e */
                    for (int e = 0; e < 3; e++) {
                        int cm[3] = {c[0], c[1], c[2]};
                        cm[e] = wrap(c[e] - 1, dims[e]);
                        int64_t im = cell_index(cm[0], cm[1], cm[2], nx, ny);
                        for (int v = 0; v < NV; v++)
                            div[e][v] = FX[((int64_t)e * NV + v) * n + i] - FX[((int64_t)e * NV + v) * n + im];
                    }
                    for (int d = 0; d < 3; d++) {
                        int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
                        for (int s2 = 0; s2 < 2; s2++)
                            for (int v = 0; v < NV; v++)
                                FS[((int64_t)(2 * d + s2) * NV + v) * n + i] -=
                                    0.5 * dt / dh * (div[e1][v] + div[e2][v]);
                    }
                }
        or_face_fluxes(FS, FX, nx, ny, nz, gamma);
    }

    /* 5. conservative update */
    int64_t nbad = 0;
#pragma omp parallel for schedule(static) reduction(+ : nbad)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int c[3] = {x, y, z};
                int64_t i = cell_index(x, y, z, nx, ny);
                double un[NV];
                for (int v = 0; v < NV; v++) {
                    double div = 0.0;
                    for (int d = 0; d < 3; d++) {
                        int cm[3] = {c[0], c[1], c[2]};
                        cm[d] = wrap(c[d] - 1, dims[d]);
                        int64_t im = cell_index(cm[0], cm[1], cm[2], nx, ny);
                        div += FX[((int64_t)d * NV + v) * n + i] - FX[((int64_t)d * NV + v) * n + im];
                    }
                    un[v] = U[v * n + i] - dt / dh * div;
                    Unew[v * n + i] = un[v];
                }
                if (or_de_S) { /* entropy update and the dual-energy choice */
                    double div = 0.0;
                    for (int d = 0; d < 3; d++) {
                        int cm[3] = {c[0], c[1], c[2]};
                        cm[d] = wrap(c[d] - 1, dims[d]);
                        int64_t im = cell_index(cm[0], cm[1], cm[2], nx, ny);
                        div += FXs[(int64_t)d * n + i] - FXs[(int64_t)d * n + im];
                    }
                    double sn = or_de_S[i] - dt / dh * div;
                    double ekin = 0.5 * (un[1] * un[1] + un[2] * un[2] + un[3] * un[3]) / un[0];
                    double eth = un[4] - ekin;
                    double rg = pow(un[0], gamma - 1.0);
                    if (eth < or_de_xi * ekin) {
                        un[4] = ekin + sn * rg / (gamma - 1.0);
                        Unew[4 * n + i] = un[4];
                    } else {
                        sn = (gamma - 1.0) * eth / rg;
                    }
                    or_de_Snew[i] = sn;
                }
                if (!or_physical(un, gamma)) {
                    int ok = 0;
                    if (or_fallback) { /* (ii), (iii) */
                        ok = or_fallback_cell(U, nx, ny, nz, x, y, z, dh, dt, gamma, un);
                        for (int v = 0; v < NV; v++) Unew[v * n + i] = un[v];
                    }
                    if (!ok) nbad++;
                }
            }

    if (FX_out) memcpy(FX_out, FX, sizeof(double) * 3 * NV * n);
    if (or_de_FXs_out && FXs) memcpy(or_de_FXs_out, FXs, sizeof(double) * 3 * n);
    free(Q);
    free(FSs);
    free(FXs);
    free(Uh);
    free(W);
    free(FS);
    free(FX);
    return nbad;
}

/* The predictor of the gravity coupling: one MUSCL-Hancock step whose half
 * step adds (dt/2) (0, rho g, m.g) of each reconstructed face state, g the
 * cell's acceleration at t^n, [3][nz][ny][nx].  Returns the unphysical
 * count, or -1 for a scheme other than MUSCL-Hancock. */
int64_t or_step_gravity_predictor(const double *U, const double *g, double *Unew, int nx, int ny, int nz, double dh,
                                  double dt, double gamma) {
    if (or_vl) return -1;
    or_grav_g = g;
    int64_t nbad = or_step_periodic_fx(U, Unew, nx, ny, nz, dh, dt, gamma, NULL);
    or_grav_g = NULL;
    return nbad;
}

/* The same predictor, also returning the face fluxes FX_out [3][5][cells]
 * through the high face of every cell (for the refined levels' flux
 * registers). */
int64_t or_step_gravity_predictor_fx(const double *U, const double *g, double *Unew, int nx, int ny, int nz,
                                     double dh, double dt, double gamma, double *FX_out) {
    if (or_vl) return -1;
    or_grav_g = g;
    int64_t nbad = or_step_periodic_fx(U, Unew, nx, ny, nz, dh, dt, gamma, FX_out);
    or_grav_g = NULL;
    return nbad;
}

/* One MUSCL-Hancock step with the dual-energy formalism: S, Snew the entropy
 * per unit volume [nz][ny][nx] before and after, xi the threshold on
 * E_the / E_kin.  Returns the unphysical count, or -1 for a scheme other
 * than MUSCL-Hancock. */
int64_t or_step_dual(const double *U, const double *S, double *Unew, double *Snew, int nx, int ny, int nz,
                     double dh, double dt, double gamma, double xi) {
    if (or_vl || or_ctu) return -1;
    or_de_S = S;
    or_de_Snew = Snew;
    or_de_xi = xi;
    int64_t nbad = or_step_periodic_fx(U, Unew, nx, ny, nz, dh, dt, gamma, NULL);
    or_de_S = NULL;
    or_de_Snew = NULL;
    return nbad;
}

/* or_step_dual that also returns the face fluxes through the high face of
 * every cell: FX_out [3][5][cells] of the conserved variables, FXs_out
 * [3][cells] of the entropy (for the refined levels' flux registers). */
int64_t or_step_dual_fx(const double *U, const double *S, double *Unew, double *Snew, int nx, int ny, int nz,
                        double dh, double dt, double gamma, double xi, double *FX_out, double *FXs_out) {
    if (or_vl || or_ctu) return -1;
    or_de_S = S;
    or_de_Snew = Snew;
    or_de_xi = xi;
    or_de_FXs_out = FXs_out;
    int64_t nbad = or_step_periodic_fx(U, Unew, nx, ny, nz, dh, dt, gamma, FX_out);
    or_de_S = NULL;
    or_de_Snew = NULL;
    or_de_FXs_out = NULL;
    return nbad;
}

/* ---- conservation sums (pairwise, fixed order) ------------------------- */

static double pairwise_sum(const double *a, int64_t n) {
    if (n <= 8) {
        double s = 0.0;
        for (int64_t i = 0; i < n; i++) s += a[i];
        return s;
    }
    int64_t h = n / 2;
    return pairwise_sum(a, h) + pairwise_sum(a + h, n - h);
}

/* out[v] = sum_cells U[v] * dV, pairwise summation in cell order. */
void or_conserved_sum(const double *U, int64_t ncell, double dV, double *out) {
    for (int v = 0; v < NV; v++) out[v] = pairwise_sum(U + v * ncell, ncell) * dV;
}

/* ---- exact Riemann solver for the 1D Euler equations (Toro 2009 ch. 4) -- */
/* Used only to validate the scheme on Sod-type problems. */

static void pressure_fn(double p, double rk, double pk, double ck, double gamma,
                        double *f, double *df) {
    if (p > pk) { /* shock */
        double A = 2.0 / ((gamma + 1.0) * rk), B = (gamma - 1.0) / (gamma + 1.0) * pk;
        double q = sqrt(A / (p + B));
        *f = (p - pk) * q;
        *df = q * (1.0 - 0.5 * (p - pk) / (B + p));
    } else { /* rarefaction */
        double e = (gamma - 1.0) / (2.0 * gamma);
        *f = 2.0 * ck / (gamma - 1.0) * (pow(p / pk, e) - 1.0);
        *df = 1.0 / (rk * ck) * pow(p / pk, -(gamma + 1.0) / (2.0 * gamma));
    }
}

/* Star pressure and velocity by Newton iteration on f(p) = fL + fR + du. */
int or_exact_star(double rl, double ul, double pl, double rr, double ur, double pr,
                  double gamma, double *pstar, double *ustar) {
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double p = 0.5 * (pl + pr); /* arithmetic-mean start, always positive */
    double fl, dfl, fr, dfr;
    for (int it = 0; it < 200; it++) {
        pressure_fn(p, rl, pl, cl, gamma, &fl, &dfl);
        pressure_fn(p, rr, pr, cr, gamma, &fr, &dfr);
        double pn = p - (fl + fr + (ur - ul)) / (dfl + dfr);
        if (pn <= 0.0) pn = 1e-14 * p;
        double change = 2.0 * fabs(pn - p) / (pn + p);
        p = pn;
        if (change < 1e-15) break;
    }
    pressure_fn(p, rl, pl, cl, gamma, &fl, &dfl);
    pressure_fn(p, rr, pr, cr, gamma, &fr, &dfr);
    *pstar = p;
    *ustar = 0.5 * (ul + ur) + 0.5 * (fr - fl);
    return 0;
}

/* Star pressure by bisection (independent check of the Newton result). */
double or_exact_pstar_bisect(double rl, double ul, double pl, double rr, double ur,
                             double pr, double gamma) {
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double lo = 1e-12, hi = 100.0 * (pl > pr ? pl : pr);
    double fl, d, fr;
    for (int it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi);
        pressure_fn(mid, rl, pl, cl, gamma, &fl, &d);
        pressure_fn(mid, rr, pr, cr, gamma, &fr, &d);
        if (fl + fr + (ur - ul) > 0.0) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* Sample the exact solution at similarity coordinates xi = x/t. */
void or_exact_sample(double rl, double ul, double pl, double rr, double ur, double pr,
                     double gamma, const double *xi, int n, double *rho, double *u,
                     double *p) {
    double ps, us;
    or_exact_star(rl, ul, pl, rr, ur, pr, gamma, &ps, &us);
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double g1 = (gamma - 1.0) / (gamma + 1.0);
    for (int i = 0; i < n; i++) {
        double s = xi[i], r, v, q;
        if (s <= us) { /* left of the contact */
            if (ps > pl) { /* left shock */
                double SL = ul - cl * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl +
                                           (gamma - 1.0) / (2.0 * gamma));
                if (s <= SL) { r = rl; v = ul; q = pl; }
                else { r = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0); v = us; q = ps; }
            } else { /* left rarefaction */
                double cs = cl * pow(ps / pl, (gamma - 1.0) / (2.0 * gamma));
                double head = ul - cl, tail = us - cs;
                if (s <= head) { r = rl; v = ul; q = pl; }
                else if (s >= tail) { r = rl * pow(ps / pl, 1.0 / gamma); v = us; q = ps; }
                else {
                    double k = 2.0 / (gamma + 1.0) + g1 / cl * (ul - s);
                    r = rl * pow(k, 2.0 / (gamma - 1.0));
                    v = 2.0 / (gamma + 1.0) * (cl + (gamma - 1.0) / 2.0 * ul + s);
                    q = pl * pow(k, 2.0 * gamma / (gamma - 1.0));
                }
            }
        } else { /* right of the contact */
            if (ps > pr) { /* right shock */
                double SR = ur + cr * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr +
                                           (gamma - 1.0) / (2.0 * gamma));
                if (s >= SR) { r = rr; v = ur; q = pr; }
                else { r = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0); v = us; q = ps; }
            } else { /* right rarefaction */
                double cs = cr * pow(ps / pr, (gamma - 1.0) / (2.0 * gamma));
                double head = ur + cr, tail = us + cs;
                if (s >= head) { r = rr; v = ur; q = pr; }
                else if (s <= tail) { r = rr * pow(ps / pr, 1.0 / gamma); v = us; q = ps; }
                else {
                    double k = 2.0 / (gamma + 1.0) - g1 / cr * (ur - s);
                    r = rr * pow(k, 2.0 / (gamma - 1.0));
                    v = 2.0 / (gamma + 1.0) * (-cr + (gamma - 1.0) / 2.0 * ur + s);
                    q = pr * pow(k, 2.0 * gamma / (gamma - 1.0));
                }
            }
        }
        rho[i] = r;
        u[i] = v;
        p[i] = q;
    }
}
