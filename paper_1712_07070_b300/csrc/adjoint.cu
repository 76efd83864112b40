// adjoint.cu -- discrete adjoint of one uniform periodic MUSCL-Hancock step
// (no counterpart in the paper: the reverse of the section 2.2 update with dt
// held fixed), lam_n = (dU^{n+1}/dU^n)^T lam_{n+1}, in FP64.
//
// The step is reversed by hand, stage by stage, over dense level-wide
// scratch arrays [component][cell]:
//   1. W = prim(U^n)                                       (per cell)
//   2. Hancock face states FS[6][5] recomputed             (per cell)
//   3. lam_F = (dt/dh)(lam_{i+1} - lam_i) at every face; HLLC VJP gives the
//      adjoints of its two face states -- every face state belongs to one
//      face, so each is written exactly once               (per cell and dim)
//   4. reverse of the Hancock cell: adjoint of the cell's own primitives and
//      of the limiter inputs a = W_i - W_{i-1}, b = W_{i+1} - W_i (per cell)
//   5. gather: each cell collects the limiter adjoints of its two
//      neighbours per dimension (no atomics: deterministic), adds the
//      identity term of U^{n+1} = U^n - ... and maps W -> U  (per cell)
// At kinks the derivative of the branch the forward evaluation takes is used
// (limiter: zero when ab <= 0; min/max of wave speeds: the selected
// argument, first on ties; HLLC: the region selected by the signs).
#include <cuda_runtime.h>

#include <vector>

#include "amr_hydro.h"
#include "ctx.h"
#include "hydro_math.cuh"

namespace {

constexpr int NV = 5;
using amrh::rcp_;   // FP64 reciprocal: special-function seed + one third-order refinement
using amrh::sqrt_;  // FP64 square root: x * refined rsqrt on positive normals
using amrh::ge0;
using amrh::le0;
using amrh::gt0;
using amrh::okey;

struct Dims {
    int nx, ny, nz;
    int64_t n;
    __device__ __forceinline__ int64_t at(int x, int y, int z) const {
        x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
        return ((int64_t)z * ny + y) * nx + x;
    }
};

__device__ __forceinline__ void prim(const double U[NV], double W[NV], double gm1) {
    const double r = U[0], ri = rcp_(r);
    const double vx = U[1] * ri, vy = U[2] * ri, vz = U[3] * ri;
    const double ek = 0.5 * r * (vx * vx + vy * vy + vz * vz);
    W[0] = r;
    W[1] = vx;
    W[2] = vy;
    W[3] = vz;
    W[4] = gm1 * (U[4] - ek);
}

// lU += (dW/dU)^T lW
__device__ __forceinline__ void prim_adj(const double U[NV], const double lW[NV], double lU[NV], double gm1) {
    const double r = U[0], ri = rcp_(r);
    const double v[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
    const double lek = -gm1 * lW[4];
    lU[4] += gm1 * lW[4];
    double lr = lW[0] + lek * 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double lv = lW[1 + k] + lek * r * v[k];
        lU[1 + k] += lv * ri;
        lr -= lv * v[k] * ri;
    }
    lU[0] += lr;
}

__device__ __forceinline__ void cons(const double W[NV], double U[NV], double inv_gm1) {
    const double r = W[0];
    U[0] = r;
    U[1] = r * W[1];
    U[2] = r * W[2];
    U[3] = r * W[3];
    U[4] = W[4] * inv_gm1 + 0.5 * r * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

// lW += (dU/dW)^T lU
__device__ __forceinline__ void cons_adj(const double W[NV], const double lU[NV], double lW[NV], double inv_gm1) {
    const double r = W[0];
    const double k2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
    lW[0] += lU[0] + lU[1] * W[1] + lU[2] * W[2] + lU[3] * W[3] + lU[4] * 0.5 * k2;
#pragma unroll
    for (int k = 0; k < 3; k++) lW[1 + k] += lU[1 + k] * r + lU[4] * r * W[1 + k];
    lW[4] += lU[4] * inv_gm1;
}

// physical flux along d of conserved U (through its primitives)
__device__ __forceinline__ void flux(const double U[NV], int d, double F[NV], double gm1) {
    double W[NV];
    prim(U, W, gm1);
    const double vn = W[1 + d], P = W[4];
    F[0] = U[0] * vn;
    F[1] = U[1] * vn;
    F[2] = U[2] * vn;
    F[3] = U[3] * vn;
    F[1 + d] += P;
    F[4] = (U[4] + P) * vn;
}

// lU += (dF/dU)^T lF
__device__ __forceinline__ void flux_adj(const double U[NV], int d, const double lF[NV], double lU[NV], double gm1) {
    double W[NV];
    prim(U, W, gm1);
    const double vn = W[1 + d], P = W[4];
    double lW[NV] = {0, 0, 0, 0, 0};
    lW[1 + d] = lF[0] * U[0] + lF[1] * U[1] + lF[2] * U[2] + lF[3] * U[3] + lF[4] * (U[4] + P);
    lW[4] = lF[1 + d] + lF[4] * vn;
    lU[0] += lF[0] * vn;
    lU[1] += lF[1] * vn;
    lU[2] += lF[2] * vn;
    lU[3] += lF[3] * vn;
    lU[4] += lF[4] * vn;
    prim_adj(U, lW, lU, gm1);
}

// (dF/dUL)^T lF and (dF/dUR)^T lF of the HLLC flux (Einfeldt/Roe outer
// speeds, contact speed S*, Toro's star states), added into lUL / lUR.
__device__ void hllc_vjp(const double UL[NV], const double UR[NV], int d, double g, const double lF[NV],
                         double lUL[NV], double lUR[NV]) {
    const double gm1 = g - 1.0;
    double WL[NV], WR[NV];
    prim(UL, WL, gm1);
    prim(UR, WR, gm1);
    const double rl = WL[0], pl = WL[4], ul = WL[1 + d];
    const double rr = WR[0], pr = WR[4], ur = WR[1 + d];
    const double ril = rcp_(rl), rir = rcp_(rr);
    const double cl = sqrt_(g * pl * ril), cr = sqrt_(g * pr * rir);
    const double sl = sqrt_(rl), sr = sqrt_(rr), S = sl + sr, iS = rcp_(S);
    double vt[3], Tk[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        Tk[k] = sl * WL[1 + k] + sr * WR[1 + k];
        vt[k] = Tk[k] * iS;
    }
    const double hl = (UL[4] + pl) * ril, hr = (UR[4] + pr) * rir;
    const double T = sl * hl + sr * hr, ht = T * iS;
    const double X = gm1 * (ht - 0.5 * (vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]));
    const double ct = sqrt_(X);
    const double a = ul - cl, b = vt[d] - ct;
    const bool selL = okey(a) <= okey(b);  // comparisons on the integer units
    const double SL = selL ? a : b;
    const double a2 = ur + cr, b2 = vt[d] + ct;
    const bool selR = okey(a2) >= okey(b2);
    const double SR = selR ? a2 : b2;
    if (ge0(SL)) {
        flux_adj(UL, d, lF, lUL, gm1);
        return;
    }
    if (le0(SR)) {
        flux_adj(UR, d, lF, lUR, gm1);
        return;
    }
    const double num = pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur);
    const double den = rl * (SL - ul) - rr * (SR - ur);
    const double iden = rcp_(den);
    const double Ss = num * iden;
    const bool left = ge0(Ss);
    const double *UK = left ? UL : UR;
    const double *WK = left ? WL : WR;
    double *lUK = left ? lUL : lUR;
    const double SK = left ? SL : SR;
    const double rK = WK[0], uK = WK[1 + d], pK = WK[4], EK = UK[4];
    const double riK = left ? ril : rir;
    const double D = rK * (SK - uK), M = SK - Ss, iM = rcp_(M), fac = D * iM;
    const double iD = rcp_(D), R = pK * iD;
    const double Q = EK * riK + (Ss - uK) * (Ss + R);
    double Us[NV];
    Us[0] = fac;
    Us[1] = fac * WK[1];
    Us[2] = fac * WK[2];
    Us[3] = fac * WK[3];
    Us[1 + d] = fac * Ss;
    Us[4] = fac * Q;

    // F = FK + SK (Us - UK)
    flux_adj(UK, d, lF, lUK, gm1);
    double lSK = 0.0, lUs[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
        lSK += lF[v] * (Us[v] - UK[v]);
        lUs[v] = SK * lF[v];
        lUK[v] -= SK * lF[v];
    }
    double lWK[NV] = {0, 0, 0, 0, 0};
    double lfac = lUs[0] + lUs[1 + d] * Ss + lUs[4] * Q;
#pragma unroll
    for (int k = 0; k < 3; k++)
        if (k != d) {
            lfac += lUs[1 + k] * WK[1 + k];
            lWK[1 + k] += lUs[1 + k] * fac;
        }
    double lSs = lUs[1 + d] * fac;
    const double lQ = lUs[4] * fac;
    // Q = EK/rK + (Ss - uK)(Ss + R)
    lUK[4] += lQ * riK;
    double lrK = -lQ * EK * riK * riK;
    lSs += lQ * ((Ss + R) + (Ss - uK));
    double luK = -lQ * (Ss + R);
    const double lR = lQ * (Ss - uK);
    const double lpK = lR * iD;
    double lD = -lR * R * iD;
    // fac = D / M
    lD += lfac * iM;
    const double lM = -lfac * fac * iM;
    lSK += lM;
    lSs -= lM;
    // D = rK (SK - uK)
    lrK += lD * (SK - uK);
    lSK += lD * rK;
    luK -= lD * rK;
    // Ss = num / den
    const double lnum = lSs * iden, lden = -lSs * Ss * iden;
    double lWL[NV] = {0, 0, 0, 0, 0}, lWR[NV] = {0, 0, 0, 0, 0};
    double lSL = 0.0, lSR = 0.0;
    lWR[4] += lnum;
    lWL[4] -= lnum;
    lWL[0] += lnum * ul * (SL - ul);
    lWL[1 + d] += lnum * rl * (SL - 2.0 * ul);
    lSL += lnum * rl * ul;
    lWR[0] -= lnum * ur * (SR - ur);
    lWR[1 + d] -= lnum * rr * (SR - 2.0 * ur);
    lSR -= lnum * rr * ur;
    lWL[0] += lden * (SL - ul);
    lSL += lden * rl;
    lWL[1 + d] -= lden * rl;
    lWR[0] -= lden * (SR - ur);
    lSR -= lden * rr;
    lWR[1 + d] += lden * rr;
    // the star side's primitives and wave speed
    double *lWKs = left ? lWL : lWR;
    lWKs[0] += lrK;
    lWKs[1 + d] += luK;
    lWKs[4] += lpK;
#pragma unroll
    for (int k = 0; k < 3; k++) lWKs[1 + k] += lWK[1 + k];
    if (left) lSL += lSK;
    else lSR += lSK;
    // SL = min(a, b), SR = max(a2, b2)
    double lvt[3] = {0, 0, 0}, lct = 0.0, lcl = 0.0, lcr = 0.0;
    if (selL) {
        lWL[1 + d] += lSL;
        lcl -= lSL;
    } else {
        lvt[d] += lSL;
        lct -= lSL;
    }
    if (selR) {
        lWR[1 + d] += lSR;
        lcr += lSR;
    } else {
        lvt[d] += lSR;
        lct += lSR;
    }
    // ct = sqrt(X), X = gm1 (ht - |vt|^2 / 2)
    const double lX = lct * 0.5 * rcp_(ct);
    const double lht = lX * gm1;
#pragma unroll
    for (int k = 0; k < 3; k++) lvt[k] -= lX * gm1 * vt[k];
    // ht = T / S, vt_k = Tk / S
    const double lT = lht * iS;
    double lS = -lht * ht * iS;
    double lsl = lT * hl, lsr = lT * hr;
    const double lhl = lT * sl, lhr = lT * sr;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double lTk = lvt[k] * iS;
        lS -= lvt[k] * vt[k] * iS;
        lsl += lTk * WL[1 + k];
        lWL[1 + k] += lTk * sl;
        lsr += lTk * WR[1 + k];
        lWR[1 + k] += lTk * sr;
    }
    lsl += lS;
    lsr += lS;
    // hl = (E + p)/rho
    lUL[4] += lhl * ril;
    lWL[4] += lhl * ril;
    lWL[0] -= lhl * hl * ril;
    lUR[4] += lhr * rir;
    lWR[4] += lhr * rir;
    lWR[0] -= lhr * hr * rir;
    // sqrt(rho)
    lWL[0] += lsl * 0.5 * rcp_(sl);
    lWR[0] += lsr * 0.5 * rcp_(sr);
    // c = sqrt(g p / rho)
    {
        const double lY = lcl * 0.5 * rcp_(cl);
        lWL[4] += lY * g * ril;
        lWL[0] -= lY * g * pl * ril * ril;
    }
    {
        const double lY = lcr * 0.5 * rcp_(cr);
        lWR[4] += lY * g * rir;
        lWR[0] -= lY * g * pr * rir * rir;
    }
    prim_adj(UL, lWL, lUL, gm1);
    prim_adj(UR, lWR, lUR, gm1);
}

__global__ void k_adj_prim(const double *__restrict__ U, double *__restrict__ W, Dims D, double gm1) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D.n; i += (int64_t)gridDim.x * blockDim.x) {
        double u[NV], w[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) u[v] = U[v * D.n + i];
        prim(u, w, gm1);
#pragma unroll
        for (int v = 0; v < NV; v++) W[v * D.n + i] = w[v];
    }
}

// Forward Hancock cell (oracle form): slopes, face states, half-step
// increment.  Outputs the six face states FS[f][v] and, for the reverse,
// the intermediates.
struct HancockCell {
    double w[NV], a[3][NV], b[3][NV], slope[3][NV], Wf[6][NV], Uf[6][NV];
};

__device__ void hancock_fwd(const double *__restrict__ W, const Dims &D, int x, int y, int z, double gamma,
                            HancockCell &H, double FS[6][NV], double c) {
    const int64_t i = D.at(x, y, z);
    const int64_t nb[3][2] = {{D.at(x - 1, y, z), D.at(x + 1, y, z)},
                              {D.at(x, y - 1, z), D.at(x, y + 1, z)},
                              {D.at(x, y, z - 1), D.at(x, y, z + 1)}};
#pragma unroll
    for (int v = 0; v < NV; v++) H.w[v] = W[v * D.n + i];
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const double a = H.w[v] - W[v * D.n + nb[d][0]];
            const double b = W[v * D.n + nb[d][1]] - H.w[v];
            H.a[d][v] = a;
            H.b[d][v] = b;
            const double ab = a * b;
            const double s = gt0(ab) ? 2.0 * ab * rcp_(a + b) : 0.0;
            H.slope[d][v] = s;
            H.Wf[2 * d][v] = H.w[v] - 0.5 * s;
            H.Wf[2 * d + 1][v] = H.w[v] + 0.5 * s;
        }
    double inc[NV] = {0, 0, 0, 0, 0};
    const double gm1 = gamma - 1.0;
    const double inv_gm1 = rcp_(gm1);
#pragma unroll
    for (int f = 0; f < 6; f++) cons(H.Wf[f], H.Uf[f], inv_gm1);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double Fm[NV], Fp[NV];
        flux(H.Uf[2 * d], d, Fm, gm1);
        flux(H.Uf[2 * d + 1], d, Fp, gm1);
#pragma unroll
        for (int v = 0; v < NV; v++) inc[v] += Fm[v] - Fp[v];
    }
#pragma unroll
    for (int f = 0; f < 6; f++)
#pragma unroll
        for (int v = 0; v < NV; v++) FS[f][v] = H.Uf[f][v] + c * inc[v];
}

__global__ void k_adj_faces_fwd(const double *__restrict__ W, double *__restrict__ FS, Dims D, double gamma,
                                double c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % D.nx), y = (int)((i / D.nx) % D.ny), z = (int)(i / ((int64_t)D.nx * D.ny));
        HancockCell H;
        double fs[6][NV];
        hancock_fwd(W, D, x, y, z, gamma, H, fs, c);
#pragma unroll
        for (int f = 0; f < 6; f++)
#pragma unroll
            for (int v = 0; v < NV; v++) FS[(f * NV + v) * D.n + i] = fs[f][v];
    }
}

// Face i+1/2 along d: lam_F = (dt/dh)(lam_{i+1} - lam_i); HLLC VJP into the
// adjoints of the high face state of cell i and the low face state of i+1.
__global__ void k_adj_hllc(const double *__restrict__ FS, const double *__restrict__ L, double *__restrict__ LFS,
                           Dims D, double gamma, double dtdh) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * D.n; t += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(t / D.n);
        const int64_t i = t % D.n;
        const int x = (int)(i % D.nx), y = (int)((i / D.nx) % D.ny), z = (int)(i / ((int64_t)D.nx * D.ny));
        const int64_t j = D.at(x + (d == 0), y + (d == 1), z + (d == 2));
        double UL[NV], UR[NV], lF[NV], lUL[NV] = {0, 0, 0, 0, 0}, lUR[NV] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int v = 0; v < NV; v++) {
            UL[v] = FS[((2 * d + 1) * NV + v) * D.n + i];
            UR[v] = FS[((2 * d) * NV + v) * D.n + j];
            lF[v] = dtdh * (L[v * D.n + j] - L[v * D.n + i]);
        }
        hllc_vjp(UL, UR, d, gamma, lF, lUL, lUR);
#pragma unroll
        for (int v = 0; v < NV; v++) {
            LFS[((2 * d + 1) * NV + v) * D.n + i] = lUL[v];
            LFS[((2 * d) * NV + v) * D.n + j] = lUR[v];
        }
    }
}

// Reverse of the Hancock cell: from the face-state adjoints to the adjoint of
// the cell's own primitives (Lself) and of its limiter inputs a, b (Lab).
__global__ void k_adj_hancock_rev(const double *__restrict__ W, const double *__restrict__ LFS,
                                  double *__restrict__ Lself, double *__restrict__ Lab, Dims D, double gamma,
                                  double c) {
    const double gm1 = gamma - 1.0, inv_gm1 = rcp_(gm1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % D.nx), y = (int)((i / D.nx) % D.ny), z = (int)(i / ((int64_t)D.nx * D.ny));
        HancockCell H;
        double fs[6][NV];
        hancock_fwd(W, D, x, y, z, gamma, H, fs, c);
        double lUf[6][NV], linc[NV] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int f = 0; f < 6; f++)
#pragma unroll
            for (int v = 0; v < NV; v++) {
                lUf[f][v] = LFS[(f * NV + v) * D.n + i];
                linc[v] += lUf[f][v];
            }
        double lincn[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            linc[v] *= c;
            lincn[v] = -linc[v];
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
            flux_adj(H.Uf[2 * d], d, linc, lUf[2 * d], gm1);
            flux_adj(H.Uf[2 * d + 1], d, lincn, lUf[2 * d + 1], gm1);
        }
        double lw[NV] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            double lm[NV] = {0, 0, 0, 0, 0}, lp[NV] = {0, 0, 0, 0, 0};
            cons_adj(H.Wf[2 * d], lUf[2 * d], lm, inv_gm1);
            cons_adj(H.Wf[2 * d + 1], lUf[2 * d + 1], lp, inv_gm1);
#pragma unroll
            for (int v = 0; v < NV; v++) {
                lw[v] += lm[v] + lp[v];
                const double ls = 0.5 * (lp[v] - lm[v]);
                const double a = H.a[d][v], b = H.b[d][v];
                double la = 0.0, lb = 0.0;
                if (gt0(a * b)) {
                    const double r = rcp_(a + b), r2 = 2.0 * ls * r * r;
                    la = r2 * b * b;
                    lb = r2 * a * a;
                }
                Lab[((d * NV + v) * 2 + 0) * D.n + i] = la;
                Lab[((d * NV + v) * 2 + 1) * D.n + i] = lb;
            }
        }
#pragma unroll
        for (int v = 0; v < NV; v++) Lself[v * D.n + i] = lw[v];
    }
}

// lam_n = lam_{n+1} + (dW/dU)^T (Lself + limiter adjoints gathered from the
// cell and its two neighbours per dimension).
__global__ void k_adj_gather(const double *__restrict__ U, const double *__restrict__ L,
                             const double *__restrict__ Lself, const double *__restrict__ Lab,
                             double *__restrict__ out, Dims D, double gm1) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % D.nx), y = (int)((i / D.nx) % D.ny), z = (int)(i / ((int64_t)D.nx * D.ny));
        double lW[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) lW[v] = Lself[v * D.n + i];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int64_t im = D.at(x - (d == 0), y - (d == 1), z - (d == 2));
            const int64_t ip = D.at(x + (d == 0), y + (d == 1), z + (d == 2));
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const int64_t base = (int64_t)(d * NV + v) * 2;
                lW[v] += Lab[base * D.n + i] - Lab[(base + 1) * D.n + i];  // a_i, b_i of this cell
                lW[v] += Lab[(base + 1) * D.n + im];                       // b_{i-1} = W_i - W_{i-1}
                lW[v] -= Lab[base * D.n + ip];                             // a_{i+1} = W_{i+1} - W_i
            }
        }
        double u[NV], lU[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) {
            u[v] = U[v * D.n + i];
            lU[v] = L[v * D.n + i];
        }
        prim_adj(u, lW, lU, gm1);
#pragma unroll
        for (int v = 0; v < NV; v++) out[v * D.n + i] = lU[v];
    }
}

__global__ void k_selftest_hllc_vjp(const double *UL, const double *UR, const double *lF, int n, int d,
                                    double gamma, double *lUL, double *lUR) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a[NV] = {0, 0, 0, 0, 0}, b[NV] = {0, 0, 0, 0, 0};
    hllc_vjp(UL + NV * i, UR + NV * i, d, gamma, lF + NV * i, a, b);
    for (int v = 0; v < NV; v++) {
        lUL[NV * i + v] = a[v];
        lUR[NV * i + v] = b[v];
    }
}

}  // namespace

using namespace amrh;

extern "C" int amrh_selftest_hllc_vjp(const double *UL, const double *UR, const double *lF, int n, int d,
                                      double gamma, double *lUL, double *lUR) {
    if (n <= 0 || d < 0 || d > 2) return 1;
    k_selftest_hllc_vjp<<<(n + 127) / 128, 128>>>(UL, UR, lF, n, d, gamma, lUL, lUR);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" amr_status amr_hydro_step_adjoint(amr_hydro_ctx *c, int level, double dt, const double *U_n,
                                             const double *lam_np1, double *lam_n) {
    if (!c || level < 0 || level > c->prm.lmax || !U_n || !lam_np1 || !lam_n) return AMR_E_INVAL;
    if (!(dt >= 0.0)) return AMR_E_INVAL;
    // the hand-written reverse covers MUSCL-Hancock with the van Leer-type limiter and HLLC
    if (c->prm.limiter != AMR_LIM_VANLEER || c->prm.riemann != AMR_RS_HLLC || c->prm.scheme != AMR_SCHEME_MH)
        return AMR_E_INVAL;
    Level &L = c->lv[level];
    const int nx = c->prm.root_n[0] << level, ny = c->prm.root_n[1] << level, nz = c->prm.root_n[2] << level;
    const int64_t n = (int64_t)nx * ny * nz;
    if ((int64_t)L.n_patches * 512 != n) return AMR_E_INVAL;  // a fully covered (uniform) level only
    // the uniform slot order of amr_hydro_uniform_tables is required
    {
        const int ngx = nx / 16, ngy = ny / 16;
        for (int s = 0; s < L.n_patches; s++) {
            const int g = s / 8, k = s % 8;
            const int gx = g % ngx, gy = (g / ngx) % ngy, gz = g / (ngx * ngy);
            if (L.corner[3 * s] != 16 * gx + 8 * (k & 1) || L.corner[3 * s + 1] != 16 * gy + 8 * ((k >> 1) & 1) ||
                L.corner[3 * s + 2] != 16 * gz + 8 * (k >> 2))
                return AMR_E_INVAL;
        }
    }
    amr_status st = c->adjbuf.reserve((size_t)n * 115);
    if (st) return st;
    double *Ud = c->adjbuf.p, *Ld = Ud + 5 * n, *Wd = Ld + 5 * n, *FS = Wd + 5 * n, *LFS = FS + 30 * n,
           *Ls = LFS + 30 * n, *Lab = Ls + 5 * n, *out = Lab + 30 * n;
    if ((st = amr_hydro_unpack_uniform(U_n, nx, ny, nz, Ud, c->stream))) return st;
    if ((st = amr_hydro_unpack_uniform(lam_np1, nx, ny, nz, Ld, c->stream))) return st;
    Dims D{nx, ny, nz, n};
    const double g = c->prm.gamma, dh = level_dh(c, level);
    const int grid = c->n_sm * 8;
    k_adj_prim<<<grid, 256, 0, c->stream>>>(Ud, Wd, D, g - 1.0);
    k_adj_faces_fwd<<<grid, 128, 0, c->stream>>>(Wd, FS, D, g, 0.5 * dt / dh);
    k_adj_hllc<<<grid, 128, 0, c->stream>>>(FS, Ld, LFS, D, g, dt / dh);
    k_adj_hancock_rev<<<grid, 128, 0, c->stream>>>(Wd, LFS, Ls, Lab, D, g, 0.5 * dt / dh);
    k_adj_gather<<<grid, 256, 0, c->stream>>>(Ud, Ld, Ls, Lab, out, D, g - 1.0);
    if ((st = cuda_fail(cudaGetLastError(), "adjoint kernels"))) return st;
    return amr_hydro_pack_uniform(out, nx, ny, nz, lam_n, c->stream);
}
