/*
 * amr_oracle.c -- FP64 CPU oracle of the AMR operations around the patch
 * update (GAMER-2 section 2.1: 8^3 patches, refinement ratio 2, flag
 * buffers; section 2.2: restriction and coarse-fine flux fix-up; section 3.2:
 * ghost zones filled by copying from siblings or interpolating from coarse
 * patches).
 *
 * TEST INFRASTRUCTURE ONLY (see hydro_oracle.c).
 *
 * Every level l is held as a dense whole-domain array U[var][z][y][x] of
 * N_l = root_n * 2^l cells per dimension, with a patch-presence mask
 * pmask[pz][py][px] (8^3-cell patches).  Only cells of present patches carry
 * the level's solution; the step of a level is the uniform periodic step of
 * hydro_oracle.c applied to the dense array after its ghost cells were filled
 * from the coarse level, of which only the present cells are kept.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV 5

static inline int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

static inline int64_t cidx(int x, int y, int z, const int N[3]) {
    return ((int64_t)z * N[1] + y) * N[0] + x;
}

static inline int patch_present(const uint8_t *pmask, const int N[3], int x, int y, int z) {
    const int P[3] = {N[0] / 8, N[1] / 8, N[2] / 8};
    int px = wrapi(x, N[0]) / 8, py = wrapi(y, N[1]) / 8, pz = wrapi(z, N[2]) / 8;
    return pmask[((int64_t)pz * P[1] + py) * P[0] + px] != 0;
}

static double minmod(double a, double b) {
    if (!(a * b > 0.0)) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* Coarse value of variable v at coarse cell (x,y,z) at the interpolation
 * time: U_old + w (U_new - U_old), exactly U_old at w = 0 and U_new at w = 1. */
static double coarse_at(const double *Uo, const double *Un, double w, int v, int x, int y, int z,
                        const int Nc[3]) {
    const int64_t n = (int64_t)Nc[0] * Nc[1] * Nc[2];
    const int64_t i = v * n + cidx(wrapi(x, Nc[0]), wrapi(y, Nc[1]), wrapi(z, Nc[2]), Nc);
    if (w == 0.0) return Uo[i];
    if (w == 1.0) return Un[i];
    return Uo[i] + w * (Un[i] - Uo[i]);
}


/*
 * Interpolated value of fine cell (x,y,z) from coarse level (C7 reading):
 * per conserved variable U_c + sum_d (+-1/4) s_d with minmod slopes of the
 * time-interpolated coarse values; if any of the eight children of the coarse
 * cell would have rho <= 0 or P <= 0 (2 rho E <= |rho v|^2), all eight take
 * U_c (slopes zeroed), which stays conservative and positive.
 */
static int interp_cell(const double *Uo, const double *Un, double w, const int Nc[3], int x, int y,
                       int z, double out[NV]) {
    const int cx = x / 2, cy = y / 2, cz = z / 2;
    double c[NV], sl[3][NV];
    for (int v = 0; v < NV; v++) {
        c[v] = coarse_at(Uo, Un, w, v, cx, cy, cz, Nc);
        sl[0][v] = minmod(coarse_at(Uo, Un, w, v, cx + 1, cy, cz, Nc) - c[v],
                          c[v] - coarse_at(Uo, Un, w, v, cx - 1, cy, cz, Nc));
        sl[1][v] = minmod(coarse_at(Uo, Un, w, v, cx, cy + 1, cz, Nc) - c[v],
                          c[v] - coarse_at(Uo, Un, w, v, cx, cy - 1, cz, Nc));
        sl[2][v] = minmod(coarse_at(Uo, Un, w, v, cx, cy, cz + 1, Nc) - c[v],
                          c[v] - coarse_at(Uo, Un, w, v, cx, cy, cz - 1, Nc));
    }
    int ok = 1;
    for (int k = 0; k < 8 && ok; k++) {
        const double sx = (k & 1) ? 0.25 : -0.25, sy = (k & 2) ? 0.25 : -0.25, sz = (k & 4) ? 0.25 : -0.25;
        double u[NV];
        for (int v = 0; v < NV; v++) u[v] = c[v] + sx * sl[0][v] + sy * sl[1][v] + sz * sl[2][v];
        const double m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
        ok = (u[0] > 0.0) && (2.0 * u[0] * u[4] > m2);
    }
    const double sx = (x & 1) ? 0.25 : -0.25, sy = (y & 1) ? 0.25 : -0.25, sz = (z & 1) ? 0.25 : -0.25;
    for (int v = 0; v < NV; v++)
        out[v] = ok ? c[v] + sx * sl[0][v] + sy * sl[1][v] + sz * sl[2][v] : c[v];
    return ok;
}

/*
 * Ghost cells of level l from level l-1 (coarse-fine interpolation).
 * Every fine cell outside the level's patches but within Chebyshev distance 3
 * of a patch cell (the ghost cells of PPM; PLM reads two) gets, per conserved
 * variable,
 *     U_f = U_c + sum_d (+-1/4) s_d,   s_d = minmod(U_{c+d} - U_c, U_c - U_{c-d}),
 * with U_c the time-interpolated coarse value of its parent cell and the sign
 * that of the child's offset from the parent centre (interp_cell, with its
 * positivity fallback).  The mean of the eight children is U_c
 * (conservative); the minmod slopes keep the children between the
 * neighbouring coarse values (monotone).  Cells farther away get a benign
 * uniform state that no stencil of a patch cell reads.
 */
void or_amr_fill_ghost(double *Uf, const uint8_t *pmask_f, const int Nf[3], const double *Uc_old,
                       const double *Uc_new, double w) {
    const int Nc[3] = {Nf[0] / 2, Nf[1] / 2, Nf[2] / 2};
    const int64_t nf = (int64_t)Nf[0] * Nf[1] * Nf[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Nf[2]; z++)
        for (int y = 0; y < Nf[1]; y++)
            for (int x = 0; x < Nf[0]; x++) {
                if (patch_present(pmask_f, Nf, x, y, z)) continue;
                int near = 0;
                for (int dz = -3; dz <= 3 && !near; dz += 3)
                    for (int dy = -3; dy <= 3 && !near; dy += 3)
                        for (int dx = -3; dx <= 3 && !near; dx += 3)
                            near = patch_present(pmask_f, Nf, x + dx, y + dy, z + dz);
                /* (the box [x-3,x+3] spans at most two patches per dimension,
                 * both reached by the offsets -3, 0, +3) */
                const int64_t i = cidx(x, y, z, Nf);
                if (!near) {
                    Uf[0 * nf + i] = 1.0;
                    Uf[1 * nf + i] = 0.0;
                    Uf[2 * nf + i] = 0.0;
                    Uf[3 * nf + i] = 0.0;
                    Uf[4 * nf + i] = 1.0;
                    continue;
                }
                double u[NV];
                interp_cell(Uc_old, Uc_new, w, Nc, x, y, z, u);
                for (int v = 0; v < NV; v++) Uf[v * nf + i] = u[v];
            }
}

/* covered[coarse cell] = 1 where level l (fine) has patches over it. */
void or_amr_covered(const uint8_t *pmask_f, const int Nf[3], uint8_t *covered) {
    const int Nc[3] = {Nf[0] / 2, Nf[1] / 2, Nf[2] / 2};
    for (int z = 0; z < Nc[2]; z++)
        for (int y = 0; y < Nc[1]; y++)
            for (int x = 0; x < Nc[0]; x++)
                covered[cidx(x, y, z, Nc)] = (uint8_t)patch_present(pmask_f, Nf, 2 * x, 2 * y, 2 * z);
}

/* Coarse-fine interface along d on the high face of coarse cell a:
 * exactly one of a, a+e_d is covered, and the uncovered one is a cell of a
 * present coarse patch. */
static int cf_face(const uint8_t *covered, const uint8_t *pmask_c, const int Nc[3], int x, int y, int z,
                   int d) {
    int b[3] = {x, y, z};
    b[d] = wrapi(b[d] + 1, Nc[d]);
    const int ca = covered[cidx(x, y, z, Nc)], cb = covered[cidx(b[0], b[1], b[2], Nc)];
    if (ca == cb) return 0;
    if (!ca) return patch_present(pmask_c, Nc, x, y, z);
    return patch_present(pmask_c, Nc, b[0], b[1], b[2]);
}

/*
 * Fine side of the flux registers (section 2.2 fix-up): after a fine step of
 * size dt_f, every coarse-fine face of the coarse level gets
 *     acc += dt_f * (mean of the 2x2 fine fluxes through it),
 * summed in a fixed order.  FXf: fine-level interface fluxes of that step,
 * [3][5][Nf cells] at the high face of every fine cell.  acc: [3][5][Nc].
 */
static void cf_fine_accumulate_nv(double *acc, const double *FXf, const uint8_t *covered, const uint8_t *pmask_c,
                                  const int Nc[3], double dt_f, int nv) {
    const int Nf[3] = {2 * Nc[0], 2 * Nc[1], 2 * Nc[2]};
    const int64_t nc = (int64_t)Nc[0] * Nc[1] * Nc[2], nf = 8 * nc;
    for (int d = 0; d < 3; d++)
        for (int z = 0; z < Nc[2]; z++)
            for (int y = 0; y < Nc[1]; y++)
                for (int x = 0; x < Nc[0]; x++) {
                    if (!cf_face(covered, pmask_c, Nc, x, y, z, d)) continue;
                    const int c[3] = {x, y, z};
                    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                    int f[3];
                    f[d] = 2 * c[d] + 1; /* fine cell whose high face is the interface */
                    for (int v = 0; v < nv; v++) {
                        double s = 0.0;
                        for (int j2 = 0; j2 < 2; j2++)
                            for (int j1 = 0; j1 < 2; j1++) {
                                f[t1] = 2 * c[t1] + j1;
                                f[t2] = 2 * c[t2] + j2;
                                s += FXf[((int64_t)d * nv + v) * nf + cidx(f[0], f[1], f[2], Nf)];
                            }
                        acc[((int64_t)d * nv + v) * nc + cidx(x, y, z, Nc)] += dt_f * (0.25 * s);
                    }
                }
}

void or_amr_cf_fine_accumulate(double *acc, const double *FXf, const uint8_t *covered,
                               const uint8_t *pmask_c, const int Nc[3], double dt_f) {
    cf_fine_accumulate_nv(acc, FXf, covered, pmask_c, Nc, dt_f, NV);
}

/* The same for the dual-energy entropy's flux (one variable: [3][Nf], [3][Nc]). */
void or_amr_cf_fine_accumulate_s(double *acc, const double *FXf, const uint8_t *covered,
                                 const uint8_t *pmask_c, const int Nc[3], double dt_f) {
    cf_fine_accumulate_nv(acc, FXf, covered, pmask_c, Nc, dt_f, 1);
}

/* Coarse side: cfl = dt_c * F_c on every coarse-fine face (0 elsewhere). */
static void cf_coarse_store_nv(double *cfl, const double *FXc, const uint8_t *covered, const uint8_t *pmask_c,
                               const int Nc[3], double dt_c, int nv) {
    const int64_t nc = (int64_t)Nc[0] * Nc[1] * Nc[2];
    for (int d = 0; d < 3; d++)
        for (int z = 0; z < Nc[2]; z++)
            for (int y = 0; y < Nc[1]; y++)
                for (int x = 0; x < Nc[0]; x++) {
                    const int64_t i = cidx(x, y, z, Nc);
                    const int on = cf_face(covered, pmask_c, Nc, x, y, z, d);
                    for (int v = 0; v < nv; v++) {
                        const int64_t k = ((int64_t)d * nv + v) * nc + i;
                        cfl[k] = on ? dt_c * FXc[k] : 0.0;
                    }
                }
}

void or_amr_cf_coarse_store(double *cfl, const double *FXc, const uint8_t *covered,
                            const uint8_t *pmask_c, const int Nc[3], double dt_c) {
    cf_coarse_store_nv(cfl, FXc, covered, pmask_c, Nc, dt_c, NV);
}

void or_amr_cf_coarse_store_s(double *cfl, const double *FXc, const uint8_t *covered,
                              const uint8_t *pmask_c, const int Nc[3], double dt_c) {
    cf_coarse_store_nv(cfl, FXc, covered, pmask_c, Nc, dt_c, 1);
}

/*
 * Flux fix-up of the leaf coarse cells next to the fine region (section 2.2):
 * across a face on the cell's high side U_c -= (acc - cfl)/dh_c, across a
 * face on its low side U_c += (acc - cfl)/dh_c; faces are applied in the
 * order -x, +x, -y, +y, -z, +z.
 */
static void fixup_nv(double *Uc, const double *acc, const double *cfl, const uint8_t *covered, const uint8_t *pmask_c,
                     const int Nc[3], double dh_c, int nv) {
    const int64_t nc = (int64_t)Nc[0] * Nc[1] * Nc[2];
    for (int z = 0; z < Nc[2]; z++)
        for (int y = 0; y < Nc[1]; y++)
            for (int x = 0; x < Nc[0]; x++) {
                const int64_t i = cidx(x, y, z, Nc);
                if (covered[i] || !patch_present(pmask_c, Nc, x, y, z)) continue;
                const int c[3] = {x, y, z};
                for (int d = 0; d < 3; d++) {
                    int m[3] = {x, y, z}, p[3] = {x, y, z};
                    m[d] = wrapi(c[d] - 1, Nc[d]);
                    p[d] = wrapi(c[d] + 1, Nc[d]);
                    const int64_t im = cidx(m[0], m[1], m[2], Nc), ip = cidx(p[0], p[1], p[2], Nc);
                    if (covered[im]) /* low face: the interface is the high face of m */
                        for (int v = 0; v < nv; v++) {
                            const int64_t k = ((int64_t)d * nv + v) * nc + im;
                            Uc[v * nc + i] += (acc[k] - cfl[k]) / dh_c;
                        }
                    if (covered[ip]) /* high face */
                        for (int v = 0; v < nv; v++) {
                            const int64_t k = ((int64_t)d * nv + v) * nc + i;
                            Uc[v * nc + i] -= (acc[k] - cfl[k]) / dh_c;
                        }
                }
            }
}

void or_amr_fixup(double *Uc, const double *acc, const double *cfl, const uint8_t *covered,
                  const uint8_t *pmask_c, const int Nc[3], double dh_c) {
    fixup_nv(Uc, acc, cfl, covered, pmask_c, Nc, dh_c, NV);
}

void or_amr_fixup_s(double *Sc, const double *acc, const double *cfl, const uint8_t *covered,
                    const uint8_t *pmask_c, const int Nc[3], double dh_c) {
    fixup_nv(Sc, acc, cfl, covered, pmask_c, Nc, dh_c, 1);
}

/* Restriction (section 2.2): every covered coarse cell becomes the mean of
 * its 8 children, summed in the order x fastest, then y, then z. */
static void restrict_nv(double *Uc, const double *Uf, const uint8_t *covered, const int Nc[3], int nv) {
    const int Nf[3] = {2 * Nc[0], 2 * Nc[1], 2 * Nc[2]};
    const int64_t nc = (int64_t)Nc[0] * Nc[1] * Nc[2], nf = 8 * nc;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Nc[2]; z++)
        for (int y = 0; y < Nc[1]; y++)
            for (int x = 0; x < Nc[0]; x++) {
                const int64_t i = cidx(x, y, z, Nc);
                if (!covered[i]) continue;
                for (int v = 0; v < nv; v++) {
                    double s = 0.0;
                    for (int dz = 0; dz < 2; dz++)
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++)
                                s += Uf[v * nf + cidx(2 * x + dx, 2 * y + dy, 2 * z + dz, Nf)];
                    Uc[v * nc + i] = s * 0.125;
                }
            }
}

void or_amr_restrict(double *Uc, const double *Uf, const uint8_t *covered, const int Nc[3]) {
    restrict_nv(Uc, Uf, covered, Nc, NV);
}

void or_amr_restrict_s(double *Sc, const double *Sf, const uint8_t *covered, const int Nc[3]) {
    restrict_nv(Sc, Sf, covered, Nc, 1);
}

/*
 * Refinement flags (section 2.1).  Cell criterion, normalised density
 * gradient: g^2 = sum_d ((rho_{+d} - rho_{-d})/2)^2 > theta^2 rho^2
 * (strict), on cells of present patches; neighbours outside the patches come
 * from the ghost-filled array.  Patch flags with the flag buffer: a present
 * patch is flagged when a flagged cell lies within Chebyshev distance nbuf of
 * one of its cells (periodic).
 */
void or_amr_flag_cells(const double *U, const uint8_t *pmask, const int N[3], double theta,
                       uint8_t *cflag) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < N[2]; z++)
        for (int y = 0; y < N[1]; y++)
            for (int x = 0; x < N[0]; x++) {
                const int64_t i = cidx(x, y, z, N);
                cflag[i] = 0;
                if (!patch_present(pmask, N, x, y, z)) continue;
                const double rho = U[i];
                const int c[3] = {x, y, z};
                double g2 = 0.0;
                for (int d = 0; d < 3; d++) {
                    int m[3] = {x, y, z}, p[3] = {x, y, z};
                    m[d] = wrapi(c[d] - 1, N[d]);
                    p[d] = wrapi(c[d] + 1, N[d]);
                    const double gd = (U[cidx(p[0], p[1], p[2], N)] - U[cidx(m[0], m[1], m[2], N)]) / 2.0;
                    g2 += gd * gd;
                }
                cflag[i] = (uint8_t)(g2 > theta * theta * (rho * rho));
            }
}

void or_amr_patch_flags(const uint8_t *cflag, const uint8_t *pmask, const int N[3], int nbuf,
                        uint8_t *pflag) {
    const int P[3] = {N[0] / 8, N[1] / 8, N[2] / 8};
#pragma omp parallel for schedule(static)
    for (int pz = 0; pz < P[2]; pz++)
        for (int py = 0; py < P[1]; py++)
            for (int px = 0; px < P[0]; px++) {
                const int64_t pi = ((int64_t)pz * P[1] + py) * P[0] + px;
                pflag[pi] = 0;
                if (!pmask[pi]) continue;
                int hit = 0;
                for (int z = 8 * pz - nbuf; z < 8 * pz + 8 + nbuf && !hit; z++)
                    for (int y = 8 * py - nbuf; y < 8 * py + 8 + nbuf && !hit; y++)
                        for (int x = 8 * px - nbuf; x < 8 * px + 8 + nbuf && !hit; x++)
                            hit = cflag[cidx(wrapi(x, N[0]), wrapi(y, N[1]), wrapi(z, N[2]), N)];
                pflag[pi] = (uint8_t)hit;
            }
}

/*
 * Data of newly created child patches (section 2.1 refinement): the children
 * of every coarse cell listed by the fine mask `newmask` (a patch mask of the
 * fine level) get the spatial interpolation of or_amr_fill_ghost from the
 * coarse state Uc (no time interpolation).
 */
void or_amr_prolong_patches(double *Uf, const uint8_t *newmask, const int Nf[3], const double *Uc) {
    const int Nc[3] = {Nf[0] / 2, Nf[1] / 2, Nf[2] / 2};
    const int64_t nf = (int64_t)Nf[0] * Nf[1] * Nf[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Nf[2]; z++)
        for (int y = 0; y < Nf[1]; y++)
            for (int x = 0; x < Nf[0]; x++) {
                if (!patch_present(newmask, Nf, x, y, z)) continue;
                const int64_t i = cidx(x, y, z, Nf);
                double u[NV];
                interp_cell(Uc, Uc, 1.0, Nc, x, y, z, u);
                for (int v = 0; v < NV; v++) Uf[v * nf + i] = u[v];
            }
}

/*
 * The dual-energy entropy per unit volume on refined levels (section 2.2
 * dual-energy formalism on the section 2.1 hierarchy): a conserved density,
 * interpolated like the conserved variables -- time first, then
 * S_f = S_c + sum_d (+-1/4) s_d with s_d = minmod(S_{c+d} - S_c, S_c - S_{c-d})
 * -- and sharing their positivity decision: where the conserved variables'
 * children fall back to the parent value (ok == 0), so does the entropy.
 */
static double interp_scalar(const double *So, const double *Sn, double w, const int Nc[3], int x, int y, int z,
                            int ok) {
    const int cx = x / 2, cy = y / 2, cz = z / 2;
    const double c = coarse_at(So, Sn, w, 0, cx, cy, cz, Nc);
    const double s0 = minmod(coarse_at(So, Sn, w, 0, cx + 1, cy, cz, Nc) - c, c - coarse_at(So, Sn, w, 0, cx - 1, cy, cz, Nc));
    const double s1 = minmod(coarse_at(So, Sn, w, 0, cx, cy + 1, cz, Nc) - c, c - coarse_at(So, Sn, w, 0, cx, cy - 1, cz, Nc));
    const double s2 = minmod(coarse_at(So, Sn, w, 0, cx, cy, cz + 1, Nc) - c, c - coarse_at(So, Sn, w, 0, cx, cy, cz - 1, Nc));
    const double sx = (x & 1) ? 0.25 : -0.25, sy = (y & 1) ? 0.25 : -0.25, sz = (z & 1) ? 0.25 : -0.25;
    return ok ? c + sx * s0 + sy * s1 + sz * s2 : c;
}

/* Entropy ghosts of level l from level l-1 (the cells or_amr_fill_ghost fills). */
void or_amr_fill_ghost_s(double *Sf, const uint8_t *pmask_f, const int Nf[3], const double *Sc_old,
                         const double *Sc_new, const double *Uc_old, const double *Uc_new, double w) {
    const int Nc[3] = {Nf[0] / 2, Nf[1] / 2, Nf[2] / 2};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Nf[2]; z++)
        for (int y = 0; y < Nf[1]; y++)
            for (int x = 0; x < Nf[0]; x++) {
                if (patch_present(pmask_f, Nf, x, y, z)) continue;
                int near = 0;
                for (int dz = -3; dz <= 3 && !near; dz += 3)
                    for (int dy = -3; dy <= 3 && !near; dy += 3)
                        for (int dx = -3; dx <= 3 && !near; dx += 3)
                            near = patch_present(pmask_f, Nf, x + dx, y + dy, z + dz);
                if (!near) {
                    Sf[cidx(x, y, z, Nf)] = 1.0;
                    continue;
                }
                double u[NV];
                const int ok = interp_cell(Uc_old, Uc_new, w, Nc, x, y, z, u);
                Sf[cidx(x, y, z, Nf)] = interp_scalar(Sc_old, Sc_new, w, Nc, x, y, z, ok);
            }
}

/* Entropy of newly created patches of the fine level, from the coarse S. */
void or_amr_prolong_patches_s(double *Sf, const uint8_t *newmask, const int Nf[3], const double *Sc,
                              const double *Uc) {
    const int Nc[3] = {Nf[0] / 2, Nf[1] / 2, Nf[2] / 2};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Nf[2]; z++)
        for (int y = 0; y < Nf[1]; y++)
            for (int x = 0; x < Nf[0]; x++)
                if (patch_present(newmask, Nf, x, y, z)) {
                    double u[NV];
                    const int ok = interp_cell(Uc, Uc, 1.0, Nc, x, y, z, u);
                    Sf[cidx(x, y, z, Nf)] = interp_scalar(Sc, Sc, 1.0, Nc, x, y, z, ok);
                }
}

/*
 * A cell-centred field (one component of the gravitational acceleration) on
 * the ghost cells of level l from level l-1 (the cells or_amr_fill_ghost
 * fills): time interpolation, then the minmod-limited linear prolongation,
 * with no positivity decision (the field has no sign constraint).
 */
void or_amr_fill_ghost_field(double *Ff, const uint8_t *pmask_f, const int Nf[3], const double *Fc_old,
                             const double *Fc_new, double w) {
    const int Nc[3] = {Nf[0] / 2, Nf[1] / 2, Nf[2] / 2};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Nf[2]; z++)
        for (int y = 0; y < Nf[1]; y++)
            for (int x = 0; x < Nf[0]; x++) {
                if (patch_present(pmask_f, Nf, x, y, z)) continue;
                int near = 0;
                for (int dz = -3; dz <= 3 && !near; dz += 3)
                    for (int dy = -3; dy <= 3 && !near; dy += 3)
                        for (int dx = -3; dx <= 3 && !near; dx += 3)
                            near = patch_present(pmask_f, Nf, x + dx, y + dy, z + dz);
                Ff[cidx(x, y, z, Nf)] = near ? interp_scalar(Fc_old, Fc_new, w, Nc, x, y, z, 1) : 0.0;
            }
}
