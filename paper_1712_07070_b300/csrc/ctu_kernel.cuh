// ctu_kernel.cuh -- the CTU march of the fused per-patch-group step (GAMER-2
// section 2.2: the corner transport upwind scheme of Colella 1990 in the
// variant with six Riemann solves per cell, as in Athena; PLM on primitive
// variables; the time step of section 2.6 Eq. CFL1 reduced on the fly).
// Included by step_kernel.cuh after the helpers it shares with the
// MUSCL-Hancock march (tile staging, tables, coarse-fine registers, solvers).
//
// One CTA marches a run of patch groups plane by plane along z as the
// MUSCL-Hancock kernel does; iteration z (-2 .. 16 len) works on plane z:
//   A  every column owner (the 256 interior columns and the 64 ring columns
//      x = -1, 16 or y = -1, 16) predicts the z face states of its cell z+1:
//      PLM states advanced by dt/2 with the z flux difference alone (the
//      normal predictor), and solves the first z flux at z+1/2 against the
//      predicted high state of cell z; the difference dF1_z of the cell's two
//      first z fluxes stays in registers;
//   B  predicted x and y face states of the 18 x 18 cells x, y = -1..16;
//   C  first x fluxes of rows -1..16 and first y fluxes of columns -1..16;
//   D  transverse correction by each column owner of its own cell: x states
//      - (dt/2dh)(dF1_y + dF1_z), y states - (dt/2dh)(dF1_z + dF1_x), z states
//      - (dt/2dh)(dF1_x + dF1_y);
//   E  final fluxes of the corrected states: x faces of rows 0..15, y faces of
//      columns 0..15 and the z face below every interior column, with the
//      coarse-fine registers;
//   F  update of cell z-1 from U^n (staged one plane ahead), its Eq. (CFL1)
//      signal speed.
// The march starts at z = -2 (the predicted z states of cell -1) and needs the
// tile planes -NG .. 16 len - 1 + NG, like the MUSCL-Hancock march.  With PPM
// (three ghost cells) the face values of a cell reach two cells instead of
// one; the ring then holds planes z-1 .. z+3 instead of z .. z+2.
#pragma once

namespace amrh {

constexpr int CE = GE + 2;  // predicted-state region: cells -1..16 along x and y

template <typename real, int NG = 2>
struct CtuSmem {
    using Geo = Tile<NG>;
    static constexpr bool DE = false;
    real W[Geo::NR][NV][Geo::TY][Geo::TX];  // primitive ring, planes z+1-S .. z+1+S (and z)
    real XS[2][NV][CE][CE];     // x face states (low, high) of cells x, y = -1..16: [.][v][y+1][x+1]
    real YS[2][NV][CE][CE];     // y face states, same layout
    real FX[NV][CE][GE + 1];    // x flux at face x-1/2 (x = 0..16) of rows y = -1..16: [v][y+1][x]
    real FY[NV][GE + 1][CE];    // y flux at face y-1/2 (y = 0..16) of columns x = -1..16: [v][y][x+1]
    alignas(16) double raw[NV][Geo::TY * Geo::TX];  // next tile plane in flight (cp.async)
    alignas(16) double uo[2][NV][COLS];   // each column's U^n one plane ahead of its update
    int nbr[2][64];
    long long cfo[2][6];
    long long cco[2][48];
    double red[MAX_WARPS];
    double dt;
};

// Normal predictor along D of tile cell (x, y) on plane zc: the reconstructed
// (PLM or PPM) face states as conserved states, each advanced by
// (dt/2dh) [F_D(U_-) - F_D(U_+)]; with GRAV (the gravity coupling's
// predictor) each also gains (dt/2) (0, rho_f ga, m_f . ga) of its
// reconstructed state, ga the cell's acceleration at t^n.
template <typename real, int D, bool GRAV = false, typename SM>
__device__ __forceinline__ void ctu_predict(const SM &S, int x, int y, int zc, real dtdh_half, const Gas<real> &g,
                                            real um[NV], real up[NV], const real *ga = nullptr,
                                            real dt_half = real(0)) {
    using G = typename SM::Geo;
    real wm[NV], wp[NV], fm[NV], fp[NV];
    face_values<real, D, (G::S == 2)>(S, x + G::OX, y + G::OY, zc, g, wm, wp);
    w2u(wm, um, g);
    w2u(wp, up, g);
    phys_flux<D>(wm, um, fm);
    phys_flux<D>(wp, up, fp);
    if constexpr (GRAV) {
        real sm[NV], sp[NV];
        sm[0] = sp[0] = real(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            sm[1 + d] = um[0] * ga[d];
            sp[1 + d] = up[0] * ga[d];
        }
        sm[4] = um[1] * ga[0] + um[2] * ga[1] + um[3] * ga[2];
        sp[4] = up[1] * ga[0] + up[2] * ga[1] + up[3] * ga[2];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const real inc = dtdh_half * (fm[v] - fp[v]);
            um[v] = (um[v] + inc) + dt_half * sm[v];
            up[v] = (up[v] + inc) + dt_half * sp[v];
        }
    } else {
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const real inc = dtdh_half * (fm[v] - fp[v]);
            um[v] += inc;
            up[v] += inc;
        }
    }
}

// Final x / y fluxes of plane z (local plane zl of the group in table slot
// ts): the x face col - 1/2 of row `row`, the y face r - 1/2 of column col,
// and the group's high faces on one warp, with the coarse-fine registers of
// patch faces (the face coordinates of the MUSCL-Hancock kernel's x_face,
// y_face and high_faces).
template <typename real, typename SM>
__device__ __forceinline__ void ctu_x_face(SM &S, const StepParams &P, double dt, int row, int col,
                                           int zl, int ts, bool cf, const Gas<real> &g) {
    real uL[NV], uR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) { uL[v] = S.XS[1][v][row + 1][col]; uR[v] = S.XS[0][v][row + 1][col + 1]; }
    face_flux<0>(uL, uR, F, g);
#pragma unroll
    for (int v = 0; v < NV; v++) S.FX[v][row + 1][col] = F[v];
    if (cf && (col & 7) == 0) {
        const int pr = (row >> 3) * 2 + (zl >> 3) * 4;
        cf_register(S, P, dt, F, 0, row, zl, ts, col == 0 ? -1 : pr, ts, pr + (col >> 3),
                    col == 0 ? S.cfo[ts][0] : -1LL);
    }
}

template <typename real, typename SM>
__device__ __forceinline__ void ctu_y_face(SM &S, const StepParams &P, double dt, int r, int col,
                                           int zl, int ts, bool cf, const Gas<real> &g) {
    real uL[NV], uR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) { uL[v] = S.YS[1][v][r][col + 1]; uR[v] = S.YS[0][v][r + 1][col + 1]; }
    face_flux<1>(uL, uR, F, g);
#pragma unroll
    for (int v = 0; v < NV; v++) S.FY[v][r][col + 1] = F[v];
    if (cf && (r & 7) == 0) {
        const int pr = (col >> 3) + (zl >> 3) * 4;
        cf_register(S, P, dt, F, 1, col, zl, ts, r == 0 ? -1 : pr, ts, pr + 2 * (r >> 3),
                    r == 0 ? S.cfo[ts][2] : -1LL);
    }
}

template <typename real, typename SM>
__device__ __forceinline__ void ctu_high_faces(SM &S, const StepParams &P, double dt, int lane, int zl,
                                               int ts, bool cf, const Gas<real> &g) {
    const int k = lane & 15, D = lane >> 4;
    real uL[NV], uR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
        uL[v] = D == 0 ? S.XS[1][v][k + 1][GE] : S.YS[1][v][GE][k + 1];
        uR[v] = D == 0 ? S.XS[0][v][k + 1][GE + 1] : S.YS[0][v][GE + 1][k + 1];
    }
    hllc_dir(uL, uR, D, F, g);
#pragma unroll
    for (int v = 0; v < NV; v++) {
        if (D == 0) S.FX[v][k + 1][GE] = F[v];
        else S.FY[v][GE][k + 1] = F[v];
    }
    if (cf) {
        const int pa = D == 0 ? 1 + (k >> 3) * 2 + (zl >> 3) * 4 : (k >> 3) + 2 + (zl >> 3) * 4;
        cf_register(S, P, dt, F, D, k, zl, ts, pa, ts, -1, S.cfo[ts][2 * D + 1]);
    }
}

// The CTU step of a run of len patch groups stacked in z (len = 1: one
// group); arguments as for step_run.
template <typename real, bool GRAV, typename SM>
__device__ __forceinline__ void ctu_run(SM &S, const StepParams &P, const int32_t *runs, int off,
                                        int first, int len, double dt, const Gas<real> &g, real &smax_r,
                                        unsigned &nbad) {
    constexpr int NT = StepCfg<real>::NT;
    static_assert(NT == COLS, "one thread per (x,y) column");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cx = tid & 15, cy = tid >> 4;  // this thread's interior column
    // the ring column of threads 0..63: x = -1 / 16 (rows 0..15), then y = -1 / 16 (columns 0..15)
    const bool has_ring = tid < 64, xring = tid < 32;
    const int rr = tid & 15, rside = (tid >> 4) & 1;
    const int rx = xring ? (rside ? GE : -1) : rr, ry = xring ? rr : (rside ? GE : -1);
    const double dtdh = dt / P.dh;
    const real dtdh_r = (real)dtdh;
    const real dtdh_half = (real)(0.5 * dt / P.dh);
    const real dt_half = (real)(0.5 * dt);  // the gravity predictor's source factor
    const int Z = GE * len;
    int gcur = run_group(runs, off, first, 0), gprev = gcur, gnext = gcur;
    unsigned cfm = 0;  // bit s: the group in table slot s touches a coarse-fine register
    if (__syncthreads_or(load_tables(S, P, 0, gcur))) cfm = 1u;
    // iteration z (from -2) reads ring planes z and z+1-S .. z+1+S (S = 1 for
    // PLM, 2 for PPM): planes -1 - S .. S - 2 are gathered now, plane S - 1
    // is staged, and the top of iteration z converts plane z + S + 1 and
    // stages plane z + S + 2
    constexpr int SZ = SM::Geo::S;
    for (int t = -1 - SZ; t <= SZ - 2; t++) load_plane<real, ST_MH>(S, P, 0, t, t, g);
    issue_plane<real>(S, P, 0, SZ - 1);

    // interior column: predicted z states of cell z (low, high), first z flux
    // at z-1/2, corrected high z state of cell z-1, flux divergence of cell
    // z-1 (minus its top z flux); ring column: predicted high z state of cell
    // z, first z flux at z-1/2
    real pz_lo[NV], pz_hi[NV], f1z[NV], cz_hi[NV], acc[NV], rz_hi[NV], rf1z[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
        pz_lo[v] = pz_hi[v] = f1z[v] = cz_hi[v] = acc[v] = rz_hi[v] = rf1z[v] = real(0);
    }

    for (int z = -2; z <= Z; z++) {
        {  // plane z+S+1 is ready to convert, plane z+S+2 to stage
            const int t1 = z + SZ + 1;
            if (t1 <= Z + SZ) {
                const int k1 = t1 < 0 ? 0 : min(t1 >> 4, len - 1);
                finish_plane<real, ST_MH>(S, k1 & 1, t1 - GE * k1, t1, g);
            }
            const int t2 = z + SZ + 2;
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
            // U^n of columns 2 tid, 2 tid + 1 at plane z, for their update in
            // the next iteration (the slot was last read two iterations ago)
            const int64_t own = (int64_t)gcur * 8;
            const int px = (2 * tid) & 15, py = (2 * tid) >> 4;
            const double *src = P.U_old + (own + (px >> 3) + 2 * (py >> 3) + 4 * (zl >> 3)) * PSLOT +
                                (zl & 7) * 64 + (py & 7) * 8 + (px & 7);
#pragma unroll
            for (int v = 0; v < NV; v++) cp_async16(&S.uo[z & 1][v][2 * tid], src + v * PV);
            cp_async_commit();
        }
        // the next run group's tables into the slot group kz - 1 used last;
        // first read when plane 16 (kz + 1) is staged, at z = 16 kz + 12
        // with PPM (the stage runs S + 2 planes ahead)
        const bool load_next = zl == TABLE_ZL && kz + 1 < len;
        bool has_next = false;
        if (load_next) {
            gnext = run_group(runs, off, first, kz + 1);
            has_next = load_tables(S, P, (kz + 1) & 1, gnext);
        }
        const bool xy = z >= -1;          // plane z's first x / y fluxes are needed
        const bool inner = z >= 0 && z < Z;

        // ---- A: predicted z states of cell z+1, first z flux at z+1/2
        real nlo[NV], nhi[NV], dz[NV], rdz[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) nlo[v] = nhi[v] = dz[v] = rdz[v] = real(0);
        if (z < Z) {
            real ga[3];
            if constexpr (GRAV) grav_at(S, P, kz & 1, cx, cy, zl + 1, ga);
            ctu_predict<real, 2, GRAV>(S, cx, cy, z + 1, dtdh_half, g, nlo, nhi, ga, dt_half);
            if (z >= -1) {
                real f[NV];
                face_flux<2>(pz_hi, nlo, f, g);
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    dz[v] = f[v] - f1z[v];
                    f1z[v] = f[v];
                }
            }
            if (has_ring) {
                real rlo[NV], rhi[NV];
                if constexpr (GRAV) grav_at(S, P, kz & 1, rx, ry, zl + 1, ga);
                ctu_predict<real, 2, GRAV>(S, rx, ry, z + 1, dtdh_half, g, rlo, rhi, ga, dt_half);
                if (z >= -1) {
                    real f[NV];
                    face_flux<2>(rz_hi, rlo, f, g);
#pragma unroll
                    for (int v = 0; v < NV; v++) {
                        rdz[v] = f[v] - rf1z[v];
                        rf1z[v] = f[v];
                    }
                }
#pragma unroll
                for (int v = 0; v < NV; v++) rz_hi[v] = rhi[v];
            }
        }

        // ---- B: predicted x / y states of the cells -1..16 of plane z
        if (xy) {
            for (int i = tid; i < 2 * CE * CE; i += NT) {
                const int D = i >= CE * CE ? 1 : 0, j = i - D * CE * CE;
                const int x = j % CE - 1, y = j / CE - 1;
                real um[NV], up[NV], ga[3];
                if constexpr (GRAV) grav_at(S, P, kz & 1, x, y, zl, ga);
                if (D == 0) {
                    ctu_predict<real, 0, GRAV>(S, x, y, z, dtdh_half, g, um, up, ga, dt_half);
#pragma unroll
                    for (int v = 0; v < NV; v++) {
                        S.XS[0][v][y + 1][x + 1] = um[v];
                        S.XS[1][v][y + 1][x + 1] = up[v];
                    }
                } else {
                    ctu_predict<real, 1, GRAV>(S, x, y, z, dtdh_half, g, um, up, ga, dt_half);
#pragma unroll
                    for (int v = 0; v < NV; v++) {
                        S.YS[0][v][y + 1][x + 1] = um[v];
                        S.YS[1][v][y + 1][x + 1] = up[v];
                    }
                }
            }
        }
        if (load_next) {  // uniform: every thread takes the same branch
            const unsigned bit = 1u << ((kz + 1) & 1);
            cfm = __syncthreads_or(has_next) ? (cfm | bit) : (cfm & ~bit);
        } else {
            __syncthreads();
        }

        // ---- C: first x fluxes of rows -1..16, first y fluxes of columns -1..16
        if (xy) {
            constexpr int NF = CE * (GE + 1);  // faces per direction
            for (int i = tid; i < 2 * NF; i += NT) {
                const int D = i >= NF ? 1 : 0, j = i - D * NF;
                const int a = j / (GE + 1) - 1, f = j % (GE + 1);  // row (x) / column (y) a, face f - 1/2
                real uL[NV], uR[NV], F[NV];
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    uL[v] = D == 0 ? S.XS[1][v][a + 1][f] : S.YS[1][v][f][a + 1];
                    uR[v] = D == 0 ? S.XS[0][v][a + 1][f + 1] : S.YS[0][v][f + 1][a + 1];
                }
                hllc_dir(uL, uR, D, F, g);
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    if (D == 0) S.FX[v][a + 1][f] = F[v];
                    else S.FY[v][f][a + 1] = F[v];
                }
            }
        }
        __syncthreads();

        // ---- D: transverse corrections, each column owner its own cell
        real cz_lo[NV], czh[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) cz_lo[v] = czh[v] = real(0);
        if (xy) {
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const real dx = S.FX[v][cy + 1][cx + 1] - S.FX[v][cy + 1][cx];
                const real dy = S.FY[v][cy + 1][cx + 1] - S.FY[v][cy][cx + 1];
                const real cz = dtdh_half * (dx + dy);
                cz_lo[v] = pz_lo[v] - cz;
                czh[v] = pz_hi[v] - cz;
                if (inner) {
                    const real cxs = dtdh_half * (dy + dz[v]);
                    S.XS[0][v][cy + 1][cx + 1] -= cxs;
                    S.XS[1][v][cy + 1][cx + 1] -= cxs;
                    const real cys = dtdh_half * (dz[v] + dx);
                    S.YS[0][v][cy + 1][cx + 1] -= cys;
                    S.YS[1][v][cy + 1][cx + 1] -= cys;
                }
            }
            if (inner && has_ring) {
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    if (xring) {  // x states of the ring cell (rx, ry): y and z transverse terms
                        const real dy = S.FY[v][ry + 1][rx + 1] - S.FY[v][ry][rx + 1];
                        const real c = dtdh_half * (dy + rdz[v]);
                        S.XS[0][v][ry + 1][rx + 1] -= c;
                        S.XS[1][v][ry + 1][rx + 1] -= c;
                    } else {      // y states: z and x transverse terms
                        const real dx = S.FX[v][ry + 1][rx + 1] - S.FX[v][ry + 1][rx];
                        const real c = dtdh_half * (rdz[v] + dx);
                        S.YS[0][v][ry + 1][rx + 1] -= c;
                        S.YS[1][v][ry + 1][rx + 1] -= c;
                    }
                }
            }
        }
        __syncthreads();

        // ---- E: final fluxes
        real fz[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) fz[v] = real(0);
        if (z >= 0) z_face(S, P, dt, cz_hi, cz_lo, cx, cy, z, len, cfm, fz, g);
        if (inner) {
            const int ts = kz & 1;
            const bool cf = (cfm >> ts) & 1u;
            ctu_x_face(S, P, dt, cy, cx, zl, ts, cf, g);
            ctu_y_face(S, P, dt, cy, cx, zl, ts, cf, g);
            if (warp == 2) ctu_high_faces(S, P, dt, lane, zl, ts, cf, g);
        }
        __syncthreads();

        // ---- F: finish cell (cx,cy,z-1), start cell (cx,cy,z)
        if (z >= 1) {
            const int zc = z - 1, zcl = zc & (GE - 1);
            const int64_t base = ((int64_t)(zl == 0 ? gprev : gcur) * 8 + (cx >> 3) + 2 * (cy >> 3) +
                                  4 * (zcl >> 3)) * PSLOT +
                                 (zcl & 7) * 64 + (cy & 7) * 8 + (cx & 7);
            real ur[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const real tot = acc[v] + fz[v];
                const double uo = S.uo[zc & 1][v][tid];
                double un;
                if constexpr (sizeof(real) == sizeof(double)) {
                    un = uo - dtdh * tot;
                    ur[v] = un;
                } else {
                    const real inc = dtdh_r * tot;
                    un = uo - f2d_bits(inc);
                    ur[v] = d2f_bits(uo) - inc;
                }
                P.U_new[base + v * PV] = un;
            }
            bool ok;
            const real s = cfl_speed(ur, g, ok, true);
            if (!ok && !fb_append(P, base)) nbad++;
            if (s > smax_r) smax_r = s;
        }
        if (inner) {
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const real dxy = (S.FX[v][cy + 1][cx + 1] - S.FX[v][cy + 1][cx]) +
                                 (S.FY[v][cy + 1][cx + 1] - S.FY[v][cy][cx + 1]);
                acc[v] = dxy - fz[v];
            }
        }
#pragma unroll
        for (int v = 0; v < NV; v++) {
            cz_hi[v] = czh[v];
            pz_lo[v] = nlo[v];
            pz_hi[v] = nhi[v];
        }
    }
    __syncthreads();  // the next run overwrites the tables and the ring
}

}  // namespace amrh
