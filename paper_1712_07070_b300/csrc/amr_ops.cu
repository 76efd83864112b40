// amr_ops.cu -- device operations between AMR levels (GAMER-2 section 2.1:
// refinement flags and flag buffers; section 2.2: restriction and coarse-fine
// flux fix-up; section 3.2: ghost zones interpolated from coarse patches).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

using namespace amrh;

namespace {

template <typename real>
__device__ __forceinline__ real minmod(real a, real b) {
    if (!(a * b > real(0))) return real(0);
    return fabs(a) < fabs(b) ? a : b;
}

// The 27 coarse patches around coarse patch P (index (dx+1)+3(dy+1)+9(dz+1),
// 13 = P itself), from the coarse level's sibling table.
__device__ __forceinline__ void load_block27(int *nb, int P, const int32_t *csib) {
    for (int k = threadIdx.x; k < 27; k += blockDim.x) nb[k] = k == 13 ? P : csib[(int64_t)P * 26 + k - (k > 13)];
}

struct CoarseView {
    const double *Uo, *Un;
    double w;
    const int *nb;  // 27 slots around the parent
    int64_t stride = PSLOT;  // doubles per slot (PV for a one-variable field)
    // offset of variable v at coarse cell c (relative to the parent's
    // origin, each coordinate in -8..15)
    __device__ __forceinline__ int64_t index(int v, int cx, int cy, int cz) const {
        const int px = cx >> 3, py = cy >> 3, pz = cz >> 3;
        int s = nb[(px + 1) + 3 * (py + 1) + 9 * (pz + 1)];
        if (s < 0) s = nb[13];  // cannot happen on a properly nested hierarchy
        return (int64_t)s * stride + v * PV + (cz & 7) * 64 + (cy & 7) * 8 + (cx & 7);
    }
    // the coarse value there, time-interpolated
    __device__ __forceinline__ double at(int v, int cx, int cy, int cz) const {
        const int64_t i = index(v, cx, cy, cz);
        if (w == 0.0) return Uo[i];
        if (w == 1.0) return Un[i];
        return Uo[i] + w * (Un[i] - Uo[i]);
    }
};

// The coarse value in the compute type at a precomputed offset i of
// variable 0 (plus v PV for variable v): FP64 as CoarseView::at; in the
// FP32-compute mode both times' values are rounded to FP32 on the integer
// units and interpolated in FP32 (wf: w rounded once).
template <typename real>
__device__ __forceinline__ real coarse_val(const CoarseView &C, float wf, int64_t i);
template <>
__device__ __forceinline__ double coarse_val<double>(const CoarseView &C, float, int64_t i) {
    if (C.w == 0.0) return C.Uo[i];
    if (C.w == 1.0) return C.Un[i];
    return C.Uo[i] + C.w * (C.Un[i] - C.Uo[i]);
}
template <>
__device__ __forceinline__ float coarse_val<float>(const CoarseView &C, float wf, int64_t i) {
    if (C.w == 0.0) return d2f_bits(C.Uo[i]);
    if (C.w == 1.0) return d2f_bits(C.Un[i]);
    const float a = d2f_bits(C.Uo[i]);
    return a + wf * (d2f_bits(C.Un[i]) - a);
}
// Offsets (variable 0) of coarse cell c and its six face neighbours
// (centre, x+, x-, y+, y-, z+, z-): within the cell's coarse patch by
// stepping 1, 8 or 64, across a patch boundary through the 27-patch table.
__device__ __forceinline__ void stencil_index(const CoarseView &C, int cx, int cy, int cz, int64_t ic[7]) {
    ic[0] = C.index(0, cx, cy, cz);
    ic[1] = (cx & 7) != 7 ? ic[0] + 1 : C.index(0, cx + 1, cy, cz);
    ic[2] = (cx & 7) != 0 ? ic[0] - 1 : C.index(0, cx - 1, cy, cz);
    ic[3] = (cy & 7) != 7 ? ic[0] + 8 : C.index(0, cx, cy + 1, cz);
    ic[4] = (cy & 7) != 0 ? ic[0] - 8 : C.index(0, cx, cy - 1, cz);
    ic[5] = (cz & 7) != 7 ? ic[0] + 64 : C.index(0, cx, cy, cz + 1);
    ic[6] = (cz & 7) != 0 ? ic[0] - 64 : C.index(0, cx, cy, cz - 1);
}
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_bits(x); }

// Fine patches interpolated from the coarse level.  Job j (GHOST_INFO ints):
// a coarse patch P and the patch position q relative to P's children (each
// -1..2; P < 0: no job), and the box of fine cells wanted (even bounds);
// output patch out_slot[j] (or j).  Each half warp takes one job (a box has
// at most 4x4x4 coarse cells, a face ghost 4x4x1, so a whole warp per job
// would leave half of it idle on the narrow FP64 pipe); one lane per coarse
// cell of the box computes its value, slopes and positivity test once and
// writes its eight children.
constexpr int INTERP_WARPS = 8;  // warps per 256-thread block, two jobs in flight each
// With So (dual energy) the entropy per unit volume is interpolated the same
// way into outS ([slot][8^3]), sharing the conserved variables' positivity
// decision.  real: the arithmetic type.  The coarse-fine ghost patches of the
// FP32-compute mode are interpolated in FP32 (they only feed its FP32 step;
// on the FP64 pipe this kernel took a sixth of an AMR root step); the state
// of new fine patches (a regrid) is interpolated in FP64 in every mode.
template <typename real>
__global__ void k_interp_patches(double *__restrict__ out, const int32_t *__restrict__ out_slot,
                                 const int32_t *__restrict__ info, int n_jobs, const double *Uo,
                                 const double *Un, double w, const int32_t *__restrict__ csib,
                                 const double *So = nullptr, const double *Sn = nullptr, double *outS = nullptr) {
    __shared__ int nbs[2 * INTERP_WARPS][27];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    int *nb = nbs[2 * warp + half];
    for (int j0 = 2 * (blockIdx.x * INTERP_WARPS + warp); j0 < n_jobs; j0 += 2 * gridDim.x * INTERP_WARPS) {
        const int j = j0 + half;
        int P = -1, qx = 0, qy = 0, qz = 0, box = 0;
        if (j < n_jobs) {
            const int32_t *I = info + (int64_t)GHOST_INFO * j;
            P = I[0];
            qx = I[1];
            qy = I[2];
            qz = I[3];
            box = I[4];
        }
        __syncwarp();  // the previous jobs' reads of nb are done
        if (P >= 0)  // P < 0: a slot filled otherwise (a regrid's copied slots)
            for (int k = hl; k < 27; k += 16) nb[k] = k == 13 ? P : csib[(int64_t)P * 26 + k - (k > 13)];
        __syncwarp();
        if (P < 0) continue;
        const int lo[3] = {box & 15, (box >> 4) & 15, (box >> 8) & 15};
        const int hi[3] = {(box >> 12) & 15, (box >> 16) & 15, (box >> 20) & 15};
        const int n[3] = {(hi[0] - lo[0]) >> 1, (hi[1] - lo[1]) >> 1, (hi[2] - lo[2]) >> 1};
        CoarseView C{Uo, Un, w, nb};
        CoarseView CS{So, Sn, w, nb, PV};
        const float wf = (float)w;
        const int64_t oslot = out_slot ? out_slot[j] : j;
        double *o = out + oslot * PSLOT;
        const int total = n[0] * n[1] * n[2];
        for (int i = hl; i < total; i += 16) {
            // local fine cell of the child (0,0,0) of this coarse cell
            const int fx = lo[0] + 2 * (i % n[0]), fy = lo[1] + 2 * ((i / n[0]) % n[1]),
                      fz = lo[2] + 2 * (i / (n[0] * n[1]));
            // coarse cell relative to the parent's origin
            const int cx = (qx * 8 + fx) >> 1, cy = (qy * 8 + fy) >> 1, cz = (qz * 8 + fz) >> 1;
            real c[NV], sl[3][NV];
            int64_t ic[7];
            stencil_index(C, cx, cy, cz, ic);
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const int64_t vo = (int64_t)v * PV;
                c[v] = coarse_val<real>(C, wf, ic[0] + vo);
                sl[0][v] = minmod(coarse_val<real>(C, wf, ic[1] + vo) - c[v], c[v] - coarse_val<real>(C, wf, ic[2] + vo));
                sl[1][v] = minmod(coarse_val<real>(C, wf, ic[3] + vo) - c[v], c[v] - coarse_val<real>(C, wf, ic[4] + vo));
                sl[2][v] = minmod(coarse_val<real>(C, wf, ic[5] + vo) - c[v], c[v] - coarse_val<real>(C, wf, ic[6] + vo));
            }
            real u[8][NV];
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const real sx = (k & 1) ? real(0.25) : real(-0.25), sy = (k & 2) ? real(0.25) : real(-0.25),
                           sz = (k & 4) ? real(0.25) : real(-0.25);
#pragma unroll
                for (int v = 0; v < NV; v++) u[k][v] = c[v] + sx * sl[0][v] + sy * sl[1][v] + sz * sl[2][v];
                const real m2 = u[k][1] * u[k][1] + u[k][2] * u[k][2] + u[k][3] * u[k][3];
                ok = ok && (u[k][0] > real(0)) && (real(2) * u[k][0] * u[k][4] > m2);
            }
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int off = (fz + (k >> 2)) * 64 + (fy + ((k >> 1) & 1)) * 8 + fx + (k & 1);
#pragma unroll
                for (int v = 0; v < NV; v++) o[v * PV + off] = to_double(ok ? u[k][v] : c[v]);
            }
            if (So) {
                int64_t is[7];
                stencil_index(CS, cx, cy, cz, is);
                const real cs = coarse_val<real>(CS, wf, is[0]);
                const real s0 = minmod(coarse_val<real>(CS, wf, is[1]) - cs, cs - coarse_val<real>(CS, wf, is[2]));
                const real s1 = minmod(coarse_val<real>(CS, wf, is[3]) - cs, cs - coarse_val<real>(CS, wf, is[4]));
                const real s2 = minmod(coarse_val<real>(CS, wf, is[5]) - cs, cs - coarse_val<real>(CS, wf, is[6]));
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const real sx = (k & 1) ? real(0.25) : real(-0.25), sy = (k & 2) ? real(0.25) : real(-0.25),
                               sz = (k & 4) ? real(0.25) : real(-0.25);
                    const int off = (fz + (k >> 2)) * 64 + (fy + ((k >> 1) & 1)) * 8 + fx + (k & 1);
                    outS[oslot * PV + off] = to_double(ok ? cs + sx * s0 + sy * s1 + sz * s2 : cs);
                }
            }
        }
    }
}

// A three-component cell field (the gravitational acceleration, [slot][3][8^3])
// on the coarse-fine ghost patches: time interpolation, then the
// minmod-limited prolongation of each component, with no positivity
// decision.  Jobs as in k_interp_patches, half a warp each.
__global__ void k_interp_vec3(double *__restrict__ out, const int32_t *__restrict__ info, int n_jobs,
                              const double *Fo, const double *Fn, double w, const int32_t *__restrict__ csib) {
    __shared__ int nbs[2 * INTERP_WARPS][27];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    int *nb = nbs[2 * warp + half];
    for (int j0 = 2 * (blockIdx.x * INTERP_WARPS + warp); j0 < n_jobs; j0 += 2 * gridDim.x * INTERP_WARPS) {
        const int j = j0 + half;
        int P = -1, qx = 0, qy = 0, qz = 0, box = 0;
        if (j < n_jobs) {
            const int32_t *I = info + (int64_t)GHOST_INFO * j;
            P = I[0];
            qx = I[1];
            qy = I[2];
            qz = I[3];
            box = I[4];
        }
        __syncwarp();
        if (P >= 0)
            for (int k = hl; k < 27; k += 16) nb[k] = k == 13 ? P : csib[(int64_t)P * 26 + k - (k > 13)];
        __syncwarp();
        if (P < 0) continue;
        const int lo[3] = {box & 15, (box >> 4) & 15, (box >> 8) & 15};
        const int hi[3] = {(box >> 12) & 15, (box >> 16) & 15, (box >> 20) & 15};
        const int n[3] = {(hi[0] - lo[0]) >> 1, (hi[1] - lo[1]) >> 1, (hi[2] - lo[2]) >> 1};
        CoarseView C{Fo, Fn, w, nb, 3 * PV};
        double *o = out + (int64_t)j * 3 * PV;
        const int total = n[0] * n[1] * n[2];
        for (int i = hl; i < total; i += 16) {
            const int fx = lo[0] + 2 * (i % n[0]), fy = lo[1] + 2 * ((i / n[0]) % n[1]),
                      fz = lo[2] + 2 * (i / (n[0] * n[1]));
            const int cx = (qx * 8 + fx) >> 1, cy = (qy * 8 + fy) >> 1, cz = (qz * 8 + fz) >> 1;
            int64_t ic[7];
            stencil_index(C, cx, cy, cz, ic);
#pragma unroll
            for (int v = 0; v < 3; v++) {
                const int64_t vo = (int64_t)v * PV;
                const double c = coarse_val<double>(C, 0.0f, ic[0] + vo);
                const double s0 = minmod(coarse_val<double>(C, 0.0f, ic[1] + vo) - c, c - coarse_val<double>(C, 0.0f, ic[2] + vo));
                const double s1 = minmod(coarse_val<double>(C, 0.0f, ic[3] + vo) - c, c - coarse_val<double>(C, 0.0f, ic[4] + vo));
                const double s2 = minmod(coarse_val<double>(C, 0.0f, ic[5] + vo) - c, c - coarse_val<double>(C, 0.0f, ic[6] + vo));
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const double sx = (k & 1) ? 0.25 : -0.25, sy = (k & 2) ? 0.25 : -0.25, sz = (k & 4) ? 0.25 : -0.25;
                    const int off = (fz + (k >> 2)) * 64 + (fy + ((k >> 1) & 1)) * 8 + fx + (k & 1);
                    o[v * PV + off] = c + sx * s0 + sy * s1 + sz * s2;
                }
            }
        }
    }
}

// Coarse-fine flux fix-up (section 2.2).  Entry e: fix[13e] = coarse leaf
// patch Q, fix[13e+1+f] = coarse register block of face f (-1: none),
// fix[13e+7+f] = the fine register block (of the refined neighbour's child
// group) of the same interface.  Faces in the order -x,+x,-y,+y,-z,+z: a
// high face subtracts (dt_f-sum - dt_c F_c)/dh, a low face adds it.
// nreg = 6 (dual energy): the registers' sixth variable fixes the entropy S.
__global__ void k_cf_fixup(double *__restrict__ U, const int64_t *__restrict__ fix, int n_fix,
                           const double *__restrict__ creg, const double *__restrict__ freg, double dh,
                           double *__restrict__ Sv = nullptr, int nreg = NV) {
    for (int e = blockIdx.x; e < n_fix; e += gridDim.x) {
        const int64_t *F = fix + 13 * (int64_t)e;
        const int64_t Q = F[0];
        for (int f = 0; f < 6; f++) {
            const int64_t co = F[1 + f], fo = F[7 + f];
            if (co >= 0) {
                const int d = f >> 1, hi = f & 1;
                for (int i = threadIdx.x; i < 64 * nreg; i += blockDim.x) {
                    const int v = i / 64, t2 = (i >> 3) & 7, t1 = i & 7;
                    const double *B = freg + fo + (int64_t)v * 256;
                    const double fsum = 0.25 * (((B[(2 * t2) * 16 + 2 * t1] + B[(2 * t2) * 16 + 2 * t1 + 1]) +
                                                 B[(2 * t2 + 1) * 16 + 2 * t1]) +
                                                B[(2 * t2 + 1) * 16 + 2 * t1 + 1]);
                    const double corr = (fsum - creg[co + (int64_t)v * 64 + t2 * 8 + t1]) / dh;
                    const int a = hi ? 7 : 0;
                    int x, y, z;
                    if (d == 0) { x = a; y = t1; z = t2; }
                    else if (d == 1) { x = t1; y = a; z = t2; }
                    else { x = t1; y = t2; z = a; }
                    double &u = v < NV ? U[Q * PSLOT + v * PV + z * 64 + y * 8 + x] : Sv[Q * PV + z * 64 + y * 8 + x];
                    u = hi ? u - corr : u + corr;
                }
            }
            __syncthreads();
        }
    }
}

// Restriction (section 2.2): entry e = (coarse patch P, its child group G);
// each coarse cell becomes the mean of its 8 children (x fastest, then y, z).
// With Sc (dual energy) the entropy per unit volume is restricted too.
__global__ void k_restrict(double *__restrict__ Uc, const double *__restrict__ Uf, const int32_t *__restrict__ list,
                           int n, double *__restrict__ Sc = nullptr, const double *__restrict__ Sf = nullptr) {
    const int nv = Sc ? NV + 1 : NV;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const int64_t P = list[2 * e], G = list[2 * e + 1];
        for (int c = threadIdx.x; c < PV; c += blockDim.x) {
            const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
            // the eight children lie in one fine patch of the group, at b + {0, 1,
            // 8, 9, 64, 65, 72, 73}: four 16-byte pairs (b even)
            const int64_t slot = 8 * G + (x >> 2) + 2 * (y >> 2) + 4 * (z >> 2);
            const int b = ((2 * z) & 7) * 64 + ((2 * y) & 7) * 8 + ((2 * x) & 7);
            for (int v = 0; v < nv; v++) {
                const double *F = v < NV ? Uf + slot * PSLOT + v * PV + b : Sf + slot * PV + b;
                const double2 a0 = __ldg(reinterpret_cast<const double2 *>(F)),
                              a1 = __ldg(reinterpret_cast<const double2 *>(F + 8)),
                              a2 = __ldg(reinterpret_cast<const double2 *>(F + 64)),
                              a3 = __ldg(reinterpret_cast<const double2 *>(F + 72));
                // the children in (z, y, x) order, summed from the first (the sum
                // from 0 differs only in the sign of an all-negative-zero sum; on
                // the narrow FP64 pipe the add saved is a ninth of the kernel)
                double s = a0.x;
                s = s + a0.y;
                s = s + a1.x;
                s = s + a1.y;
                s = s + a2.x;
                s = s + a2.y;
                s = s + a3.x;
                s = s + a3.y;
                if (v < NV) Uc[P * PSLOT + v * PV + c] = s * 0.125;
                else Sc[P * PV + c] = s * 0.125;
            }
        }
    }
}

// The refinement criterion of one cell from its density r and the six face
// neighbours' (p: +d, m: -d): with the undivided differences d = 2 g every
// term is 4 times the criterion's, and scaling by 4 is exact, so
// D2 = dx^2 + dy^2 + dz^2 > (4 theta^2) r^2 decides exactly as
// g^2 > theta^2 r^2.  First in FP32 (values rounded on the integer units)
// with a bound on its error: every rounded value is within 2^-24 of its own
// size, each difference within delta = 2^-21 M of the exact one (M the
// largest of the seven magnitudes), so |D2_32 - D2| <= 2^-21 D2_32
// + 2 delta sum|d| + 3 delta^2 and |T_32 - T| <= 2^-20 T_32; beyond twice
// those bounds (plus the rounding of the comparison itself) the FP32 result
// is the FP64 one.  Otherwise, and for magnitudes outside [2^-40, 2^60] or
// non-finite values, the decision is taken in FP64 (the test on the bit
// patterns: both sides >= +0, a NaN flags nothing).  theta4 = 4 theta^2.
__device__ __forceinline__ bool flag_cell(double r, double px, double mx, double py, double my, double pz, double mz,
                                          double theta4, float theta4f) {
    const float rf = d2f_bits(r), pxf = d2f_bits(px), mxf = d2f_bits(mx), pyf = d2f_bits(py), myf = d2f_bits(my),
                pzf = d2f_bits(pz), mzf = d2f_bits(mz);
    const float M = fmaxf(fmaxf(fmaxf(fabsf(rf), fabsf(pxf)), fmaxf(fabsf(mxf), fabsf(pyf))),
                          fmaxf(fmaxf(fabsf(myf), fabsf(pzf)), fabsf(mzf)));
    if (M >= 9.09494702e-13f && M <= 1.1529215e18f) {  // 2^-40 .. 2^60 (NaN fails both): no square underflows
        const float dx = pxf - mxf, dy = pyf - myf, dz = pzf - mzf;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float t = theta4f * (rf * rf);
        const float delta = 4.76837158e-7f * M;  // 2^-21 M
        const float ed = 4.76837158e-7f * d2 + 2.0f * delta * (fabsf(dx) + fabsf(dy) + fabsf(dz)) + 3.0f * delta * delta;
        // + 2^-20 T, + the comparison's rounding, + 2^-120 for any flushed tiny term
        const float e = ed + 9.53674316e-7f * t + 9.53674316e-7f * (d2 + t) + 7.52316385e-37f;
        const float diff = d2 - t;
        if (diff > 2.0f * e) return true;
        if (-diff > 2.0f * e) return false;
    }
    const double ddx = px - mx, ddy = py - my, ddz = pz - mz;
    double d2 = ddx * ddx;
    d2 += ddy * ddy;
    d2 += ddz * ddz;
    const long long bd = __double_as_longlong(d2), bt = __double_as_longlong(theta4 * (r * r));
    return bd > bt && bd <= 0x7ff0000000000000LL;
}

// Cell flags (section 2.1 refinement criterion, decided as in FP64 in every
// mode, flag_cell):
// sum_d ((rho_{+d} - rho_{-d})/2)^2 > theta^2 rho^2; neighbours through the
// group's 4x4x4 source table (same-level or interpolated ghost patches).
// The cell flags themselves are not stored: each patch keeps a 27-bit
// summary of where its flagged cells lie for the flag buffer of width nbuf
// (<= 8).  Per dimension a cell is in the low part (coordinate < nbuf), the
// whole patch, and the high part (coordinate >= 8 - nbuf); bit
// a + 3 b + 9 c (a, b, c = 0 low, 1 whole, 2 high along x, y, z) is set when
// a flagged cell lies in that product of parts.  One warp per patch.
__global__ void k_flag_summary(const double *__restrict__ U, const double *__restrict__ ghost,
                               const int32_t *__restrict__ nbr, int n_groups, double theta, int nbuf,
                               uint32_t *__restrict__ summary) {
    __shared__ int src[64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;  // warp = local patch 0..7
    const double theta4 = 4.0 * (theta * theta);
    const float theta4f = d2f_bits(theta4);
    for (int g = blockIdx.x; g < n_groups; g += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < 64) src[threadIdx.x] = nbr[(int64_t)g * 64 + threadIdx.x];
        __syncthreads();
        auto rho_at = [&](int x, int y, int z) -> double {
            const int q = ((x + 8) >> 3) + 4 * ((y + 8) >> 3) + 16 * ((z + 8) >> 3);
            const int s = src[q];
            const int off = ((z + 8) & 7) * 64 + ((y + 8) & 7) * 8 + ((x + 8) & 7);
            if (s >= 0) return U[(int64_t)s * PSLOT + off];
            if (s <= -2) return ghost[(int64_t)(-2 - s) * PSLOT + off];
            return 1.0;  // a corner position: the +-1 stencil never reaches it
        };
        const int ox = 8 * (warp & 1), oy = 8 * ((warp >> 1) & 1), oz = 8 * (warp >> 2);
        uint32_t bits = 0;
        for (int c = lane; c < PV; c += 32) {
            const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
            const int x = ox + lx, y = oy + ly, z = oz + lz;
            if (!flag_cell(rho_at(x, y, z), rho_at(x + 1, y, z), rho_at(x - 1, y, z), rho_at(x, y + 1, z),
                           rho_at(x, y - 1, z), rho_at(x, y, z + 1), rho_at(x, y, z - 1), theta4, theta4f))
                continue;
            // parts this cell is in, per dimension (bit 0 low, 1 whole, 2 high)
            const int px = (lx < nbuf) | 2 | (lx >= 8 - nbuf) << 2;
            const int py = (ly < nbuf) | 2 | (ly >= 8 - nbuf) << 2;
            const int pz = (lz < nbuf) | 2 | (lz >= 8 - nbuf) << 2;
            for (int k = 0; k < 27; k++)
                if ((px >> (k % 3)) & (py >> ((k / 3) % 3)) & (pz >> (k / 9)) & 1) bits |= 1u << k;
        }
        bits = __reduce_or_sync(0xffffffffu, bits);
        if (lane == 0) summary[8 * (int64_t)g + warp] = bits;
    }
}

// Test hook kernel: flag_cell and the plain FP64 decision of n stencils
// (7 densities each: r, +x, -x, +y, -y, +z, -z).
__global__ void k_flag_cells_test(const double *__restrict__ v, int n, double theta, int *__restrict__ out) {
    const double theta4 = 4.0 * (theta * theta);
    const float theta4f = d2f_bits(theta4);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double *q = v + 7 * (int64_t)i;
        const bool f = flag_cell(q[0], q[1], q[2], q[3], q[4], q[5], q[6], theta4, theta4f);
        const double dx = q[1] - q[2], dy = q[3] - q[4], dz = q[5] - q[6];
        double d2 = dx * dx;
        d2 += dy * dy;
        d2 += dz * dz;
        const long long bd = __double_as_longlong(d2), bt = __double_as_longlong(theta4 * (q[0] * q[0]));
        const bool e = bd > bt && bd <= 0x7ff0000000000000LL;
        out[2 * i] = f;
        out[2 * i + 1] = e;
    }
}

// Patch flags with the flag buffer: patch P is flagged when a flagged cell of
// P or of a sibling lies within Chebyshev distance nbuf (<= 8) of P, that is,
// in the part of the sibling Q at offset d that faces P (along each
// dimension: Q's high part when Q lies below P, all of it when level, its
// low part when above).
__global__ void k_flag_patches(const uint32_t *__restrict__ summary, const int32_t *__restrict__ sib,
                               int n_patches, uint8_t *__restrict__ pflag) {
    for (int P = blockIdx.x * blockDim.x + threadIdx.x; P < n_patches; P += gridDim.x * blockDim.x) {
        int hit = 0;
        for (int k = 0; k < 27 && !hit; k++) {
            const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
            const int Q = k == 13 ? P : sib[(int64_t)P * 26 + k - (k > 13)];
            if (Q < 0) continue;
            const int bit = (1 - dx) + 3 * (1 - dy) + 9 * (1 - dz);
            hit = (summary[Q] >> bit) & 1u;
        }
        pflag[P] = (uint8_t)hit;
    }
}

// Per-patch sums of the conserved variables (fixed-order tree in the block).
__global__ void k_patch_sums(const double *__restrict__ U, int n_patches, double *__restrict__ out) {
    __shared__ double red[NV][256];
    for (int P = blockIdx.x; P < n_patches; P += gridDim.x) {
        double s[NV] = {0, 0, 0, 0, 0};
        for (int c = threadIdx.x; c < PV; c += 256)
#pragma unroll
            for (int v = 0; v < NV; v++) s[v] += U[(int64_t)P * PSLOT + v * PV + c];
#pragma unroll
        for (int v = 0; v < NV; v++) red[v][threadIdx.x] = s[v];
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if (threadIdx.x < h)
#pragma unroll
                for (int v = 0; v < NV; v++) red[v][threadIdx.x] += red[v][threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x < NV) out[(int64_t)P * NV + threadIdx.x] = red[threadIdx.x][0];
        __syncthreads();
    }
}

// dst[s] = src[map[s]] for every slot s with map[s] >= 0 (width doubles per slot).
// dst and src may be one buffer when no copied slot is also written.
__global__ void k_copy_slots(double *__restrict__ dst, const double *__restrict__ src,
                             const int32_t *__restrict__ map, int n, int width) {
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        const int m = map[s];
        if (m < 0) continue;
        for (int i = threadIdx.x; i < width; i += blockDim.x) dst[(int64_t)s * width + i] = src[(int64_t)m * width + i];
    }
}

}  // namespace

namespace amrh {

// time weight of the coarse level at fine time t
static double coarse_weight(const Level &C, double t) {
    if (C.t == C.t_prev || t == C.t) return 1.0;
    return (t - C.t_prev) / (C.t - C.t_prev);
}

amr_status fill_ghost_impl(amr_hydro_ctx *c, int level, double t) {
    Level &L = c->lv[level];
    if (!L.n_ghost) return AMR_OK;
    if (level == 0) return AMR_E_NESTING;
    Level &C = c->lv[level - 1];
    // the ghosts already hold this interpolation: same time, same coarse data, same plan
    if (L.ghost_valid && L.ghost_t == t && L.ghost_cver == C.version && L.ghost_pver == L.plan_version)
        return AMR_OK;
    amr_status st = level_time(c, level - 1);
    if (st) return st;
    const double w = coarse_weight(C, t);
    const int blocks = (L.n_ghost + 2 * INTERP_WARPS - 1) / (2 * INTERP_WARPS);
    const int grid = blocks < 8 * c->n_sm ? blocks : 8 * c->n_sm;
    const bool de = c->prm.dual_energy && L.ghost_S.p;
    if (c->prm.prec == AMR_FP32_ACC64)
        k_interp_patches<float><<<grid, 256, 0, c->stream>>>(
            L.ghost.p, nullptr, L.ghost_info.p, L.n_ghost, C.U[1 - C.cur], C.U[C.cur], w, C.d_sib,
            de ? C.S[1 - C.cur] : nullptr, de ? C.S[C.cur] : nullptr, de ? L.ghost_S.p : nullptr);
    else
        k_interp_patches<double><<<grid, 256, 0, c->stream>>>(
            L.ghost.p, nullptr, L.ghost_info.p, L.n_ghost, C.U[1 - C.cur], C.U[C.cur], w, C.d_sib,
            de ? C.S[1 - C.cur] : nullptr, de ? C.S[C.cur] : nullptr, de ? L.ghost_S.p : nullptr);
    if ((st = cuda_fail(cudaGetLastError(), "k_interp_patches"))) return st;
    L.ghost_valid = true;
    L.ghost_t = t;
    L.ghost_cver = C.version;
    L.ghost_pver = L.plan_version;
    return AMR_OK;
}

// g^n of a refined level's coarse-fine ghost patches at time t from the coarse
// level's accelerations at its two newest times (self-gravity in the W-cycle).
amr_status fill_ghost_acc(amr_hydro_ctx *c, int level, double t) {
    Level &L = c->lv[level];
    if (!L.n_ghost) return AMR_OK;
    if (level == 0) return AMR_E_NESTING;
    Level &C = c->lv[level - 1];
    amr_status st = level_time(c, level - 1);
    if (st) return st;
    if ((st = L.ghost_acc.reserve((size_t)L.n_ghost * 3 * PV))) return st;
    const double w = coarse_weight(C, t);
    const int blocks = (L.n_ghost + 2 * INTERP_WARPS - 1) / (2 * INTERP_WARPS);
    const int grid = blocks < 8 * c->n_sm ? blocks : 8 * c->n_sm;
    k_interp_vec3<<<grid, 256, 0, c->stream>>>(L.ghost_acc.p, L.ghost_info.p, L.n_ghost, C.gacc[1 - C.gc].p,
                                               C.gacc[C.gc].p, w, C.d_sib);
    return cuda_fail(cudaGetLastError(), "k_interp_vec3");
}

amr_status interp_new_patches(amr_hydro_ctx *c, int coarse, double *out, const int32_t *out_slot,
                              const int32_t *info, int n_jobs, double *out_S) {
    if (!n_jobs) return AMR_OK;
    Level &C = c->lv[coarse];
    const int blocks = (n_jobs + 2 * INTERP_WARPS - 1) / (2 * INTERP_WARPS);
    const int grid = blocks < 8 * c->n_sm ? blocks : 8 * c->n_sm;
    const double *cs = out_S ? C.S[C.cur] : nullptr;
    k_interp_patches<double><<<grid, 256, 0, c->stream>>>(out, out_slot, info, n_jobs, C.U[C.cur], C.U[C.cur], 1.0,
                                                   C.d_sib, cs, cs, out_S);
    return cuda_fail(cudaGetLastError(), "k_interp_patches (new patches)");
}

amr_status copy_slots(amr_hydro_ctx *c, double *dst, const double *src, const int32_t *map, int n, int width) {
    if (!n) return AMR_OK;
    const int grid = n < 8 * c->n_sm ? n : 8 * c->n_sm;
    k_copy_slots<<<grid, 256, 0, c->stream>>>(dst, src, map, n, width);
    return cuda_fail(cudaGetLastError(), "k_copy_slots");
}

amr_status patch_flags_dev(amr_hydro_ctx *c, int level, uint8_t *pflag) {
    Level &L = c->lv[level];
    amr_status st;
    if (L.n_ghost && (st = fill_ghost_impl(c, level, L.t))) return st;
    if ((st = c->flag_summary.reserve((size_t)L.n_patches))) return st;
    int nbuf = c->prm.nbuf[level];
    if (nbuf < 0) nbuf = 0;
    if (nbuf > 8) nbuf = 8;
    const int g1 = L.n_groups < 8 * c->n_sm ? L.n_groups : 8 * c->n_sm;
    k_flag_summary<<<g1, 256, 0, c->stream>>>(L.U[L.cur], L.ghost.p, L.nbr.p, L.n_groups, c->prm.theta, nbuf,
                                              c->flag_summary.p);
    if ((st = cuda_fail(cudaGetLastError(), "k_flag_summary"))) return st;
    const int g2 = (L.n_patches + 255) / 256 < 8 * c->n_sm ? (L.n_patches + 255) / 256 : 8 * c->n_sm;
    k_flag_patches<<<g2 > 0 ? g2 : 1, 256, 0, c->stream>>>(c->flag_summary.p, L.d_sib, L.n_patches, pflag);
    return cuda_fail(cudaGetLastError(), "k_flag_patches");
}

}  // namespace amrh

extern "C" {

amr_status amr_hydro_fill_ghost(amr_hydro_ctx *c, int level, double t) {
    if (!c || level <= 0 || level > c->prm.lmax) return AMR_E_INVAL;
    if (!c->lv[level].n_patches) return AMR_E_INVAL;
    return fill_ghost_impl(c, level, t);
}

amr_status amr_hydro_flux_fixup(amr_hydro_ctx *c, int l) {
    if (!c || l < 0 || l >= c->prm.lmax) return AMR_E_INVAL;
    Level &C = c->lv[l], &F = c->lv[l + 1];
    if (!C.n_patches || !F.n_patches) return AMR_OK;
    amr_status st;
    if (C.n_fix) {
        const int grid = C.n_fix < 4 * c->n_sm ? C.n_fix : 4 * c->n_sm;
        k_cf_fixup<<<grid, 128, 0, c->stream>>>(C.U[C.cur], C.fix_list.p, C.n_fix, C.creg.p, F.freg.p, level_dh(c, l),
                                                 c->prm.dual_energy ? C.S[C.cur] : nullptr, reg_vars(c));
        if ((st = cuda_fail(cudaGetLastError(), "k_cf_fixup"))) return st;
    }
    if (C.n_restrict) {
        const int grid = C.n_restrict < 8 * c->n_sm ? C.n_restrict : 8 * c->n_sm;
        k_restrict<<<grid, 256, 0, c->stream>>>(C.U[C.cur], F.U[F.cur], C.restrict_list.p, C.n_restrict,
                                                 c->prm.dual_energy ? C.S[C.cur] : nullptr,
                                                 c->prm.dual_energy ? F.S[F.cur] : nullptr);
        if ((st = cuda_fail(cudaGetLastError(), "k_restrict"))) return st;
    }
    C.speed_valid = false;
    C.version++;
    return AMR_OK;
}

amr_status amr_hydro_regrid_flags(amr_hydro_ctx *c, int level, uint8_t *flags) {
    if (!c || !flags || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    if (!c->lv[level].n_patches) return AMR_E_INVAL;
    return patch_flags_dev(c, level, flags);
}

amr_status amr_hydro_conserved_sum(amr_hydro_ctx *c, int level, double *out) {
    if (!c || !out || level < 0 || level > c->prm.lmax) return AMR_E_INVAL;
    Level &L = c->lv[level];
    for (int v = 0; v < NV; v++) out[v] = 0.0;
    if (!L.n_patches) return AMR_OK;
    amr_status st;
    if ((st = refresh_host_tables(c, level))) return st;  // leaf test on the host child table
    if ((st = c->psum.reserve((size_t)L.n_patches * NV))) return st;
    const int grid = L.n_patches < 8 * c->n_sm ? L.n_patches : 8 * c->n_sm;
    k_patch_sums<<<grid, 256, 0, c->stream>>>(L.U[L.cur], L.n_patches, c->psum.p);
    if ((st = cuda_fail(cudaGetLastError(), "k_patch_sums"))) return st;
    std::vector<double> h((size_t)L.n_patches * NV);
    if ((st = cuda_fail(cudaMemcpyAsync(h.data(), c->psum.p, 8 * h.size(), cudaMemcpyDeviceToHost, c->stream), "d2h")))
        return st;
    if ((st = cuda_fail(cudaStreamSynchronize(c->stream), "sync"))) return st;
    const double dV = level_dh(c, level) * level_dh(c, level) * level_dh(c, level);
    for (int s = 0; s < L.n_patches; s++) {
        if (L.child[s] >= 0) continue;  // covered by the finer level: not a leaf
        for (int v = 0; v < NV; v++) out[v] += h[(size_t)s * NV + v];
    }
    for (int v = 0; v < NV; v++) out[v] *= dV;
    return AMR_OK;
}

}  // extern "C"

// Test hook (not part of the C ABI): flag_cell's decisions and the plain
// FP64 ones for n host stencils (7 densities each) into out[2 i], out[2 i + 1].
// 0 on success, -1 on a CUDA error.
extern "C" int amrh_selftest_flag_cells(const double *vals, int n, double theta, int *out) {
    double *dv = nullptr;
    int *dout = nullptr;
    if (cudaMalloc(&dv, 56 * (size_t)n) != cudaSuccess) return -1;
    if (cudaMalloc(&dout, 8 * (size_t)n) != cudaSuccess) {
        cudaFree(dv);
        return -1;
    }
    int rc = 0;
    if (cudaMemcpy(dv, vals, 56 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) rc = -1;
    if (!rc) {
        k_flag_cells_test<<<(n + 255) / 256, 256>>>(dv, n, theta, dout);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(out, dout, 8 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = -1;
    }
    cudaFree(dv);
    cudaFree(dout);
    return rc;
}
