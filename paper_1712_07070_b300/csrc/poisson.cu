// poisson.cu -- GAMER-2 gravity solvers (section 2.3; section 3.1 and
// Appendix A for the refined levels): the root level's periodic or isolated
// potential by FFT, the refined levels' potential by SOR on an 18^3 grid per
// patch (the parent potential interpolated in space and, optionally, in
// time), the cell-centred accelerations, and the corrector of the
// predictor-corrector coupling of gravity to the hydro step (the predictor
// is the step kernel's ST_MH_GRAV / ST_CTU_GRAV instance).  FP64, or FP32
// transforms and SOR in the FP32-compute mode.
//
// Root level: the 7-point discrete Poisson equation
//     sum_d (phi_{i+e_d} - 2 phi_i + phi_{i-e_d}) / dh^2 = 4 pi G (rho_i - <rho>)
// is diagonal in Fourier space: phi_k = 4 pi G dh^2 rho_k / lambda_k with
// lambda_k = -2 sum_d (1 - cos(2 pi k_d / N_d)) and phi_0 = 0 (our own
// transforms, fft.cu, with the Green's factor applied between the forward
// and inverse z transforms).
//
// Isolated root level: every cell a point mass, the pairwise potential by a
// zero-padded FFT convolution with the kernel -dh^2 / |offset| (details at
// root_isolated).
//
// Refined levels: one CTA per patch holds the potential and the density of
// the patch's (8 + 2*5)^3 grid in shared memory (93 KB FP64: two CTAs per
// SM; 62 KB FP32 with padded rows: three).
// The density is the level's where a same-level patch holds the cell, else
// the parent level's cell (injection); the potential's outermost layer (held
// fixed) and initial guess come from the parent level's potential by
// quadratic interpolation in space (the tensor product of the 1-D quadratic
// through coarse cells c-1, c, c+1 at the child's offset -1/4 or +1/4, along
// x, then y, then z).  Then a fixed number of red-black SOR iterations
//     phi += omega (sum of the 6 neighbours - 6 phi - dh^2 4 pi G rho) / 6
// (red: i+j+k even in grid indices), the active 8^3 cells' potential and
// -grad phi by two- or four-point central differences.  The parent level
// holds every coarse cell read: a patch is refined only when all 26 of its
// sibling positions hold patches, and the grid reaches at most 4 coarse cells
// beyond the parent.
#include <cuda_runtime.h>

#include <cstdio>

#include "amr_hydro.h"
#include "ctx.h"
#include "fft.h"
#include "step_kernel.cuh"

namespace amrh {

namespace {

constexpr int PN = 18, PB = 5;  // SOR grid edge, buffer cells per side
constexpr int PN3 = PN * PN * PN;
constexpr double PI = 3.14159265358979323846;
constexpr double FOUR_PI = 4.0 * PI;
constexpr int SOR_NT = 256;

// ---- root level ------------------------------------------------------------------

// Deterministic sum of a block's values (256 threads): fixed shuffle pattern,
// then the 8 warp sums in order.
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
    return t;
}

// per-block partial sums of rho over the level (the mean of the source term)
__global__ void __launch_bounds__(256) k_rho_partial(const double *__restrict__ U, int n_patches,
                                                     double *__restrict__ partial) {
    __shared__ double red[8];
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n_patches * PV;
         i += (int64_t)gridDim.x * blockDim.x)
        m += U[(i / PV) * PSLOT + i % PV];
    m = block_sum(m, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = m;
}

// rho - <rho> (variable 0 of the level's current state) into a dense
// [nz][ny][nx] array of the transform's precision T; every block forms the
// same mean from the partial sums
template <typename T>
__global__ void __launch_bounds__(256) k_rho_dense(const double *__restrict__ U, const int32_t *__restrict__ corner,
                                                   int n_patches, int nx, int ny, const double *__restrict__ partial,
                                                   int n_partial, T *__restrict__ out) {
    __shared__ double red[8];
    double m = 0.0;
    for (int k = threadIdx.x; k < n_partial; k += blockDim.x) m += partial[k];
    const double mean = block_sum(m, red) / ((double)n_patches * PV);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n_patches * PV;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / PV;
        const int c = (int)(i % PV);
        const int x = corner[3 * s] + (c & 7), y = corner[3 * s + 1] + ((c >> 3) & 7),
                  z = corner[3 * s + 2] + (c >> 6);
        out[((int64_t)z * ny + y) * nx + x] = (T)(U[s * PSLOT + c] - mean);
    }
}

// The per-axis parts of the eigenvalues, lam1[k] = -2 (1 - cos(2 pi k / N)),
// for x (nx/2+1 entries), then y (ny), then z (nz).
__global__ void k_green_axes(double *__restrict__ lam1, int nx, int ny, int nz) {
    const int nxh = nx / 2 + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nxh + ny + nz; i += gridDim.x * blockDim.x) {
        int k, n;
        if (i < nxh) {
            k = i;
            n = nx;
        } else if (i < nxh + ny) {
            k = i - nxh;
            n = ny;
        } else {
            k = i - nxh - ny;
            n = nz;
        }
        lam1[i] = -2.0 * (1.0 - cos(2.0 * PI * k / n));
    }
}

// ---- isolated boundaries: zero-padded convolution with the point-mass kernel ------

// The smallest integer >= n whose prime factors are 2, 3, 5 or 7 (a size our
// transforms take with radix 2-7 stages).
int smooth7(int n) {
    for (;; n++) {
        int k = n;
        for (int p : {2, 3, 5, 7})
            while (k % p == 0) k /= p;
        if (k == 1) return n;
    }
}

// [a, a + na) and [b, b + nb) (doubles) overlap
bool overlaps(const double *a, int64_t na, const double *b, int64_t nb) {
    return a && b && a < b + nb && b < a + na;
}

int smooth7_even(int n) {
    for (n = smooth7(n); n % 2; n = smooth7(n + 1)) {
    }
    return n;
}

// The kernel -dh^2 / |offset in cells| (G = 1, cell mass rho dh^3) on the padded
// [mz][my][mx] grid, offsets wrapped to (-m/2, m/2], 0 at offset 0.
template <typename T>
__global__ void k_iso_kernel(T *__restrict__ g, int mx, int my, int mz, double dh) {
    const int64_t n = (int64_t)mx * my * mz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)(i / ((int64_t)mx * my));
        if (x > mx / 2) x -= mx;
        if (y > my / 2) y -= my;
        if (z > mz / 2) z -= mz;
        const double d = sqrt((double)x * x + (double)y * y + (double)z * z);
        g[i] = (T)(d > 0.0 ? -dh * dh / d : 0.0);
    }
}

// rho (variable 0 of the level's current state) into the first octant of the
// zeroed padded [mz][my][mx] array
template <typename T>
__global__ void k_rho_scatter(const double *__restrict__ U, const int32_t *__restrict__ corner, int n_patches,
                              int mx, int my, T *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n_patches * PV;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / PV;
        const int c = (int)(i % PV);
        const int x = corner[3 * s] + (c & 7), y = corner[3 * s + 1] + ((c >> 3) & 7),
                  z = corner[3 * s + 2] + (c >> 6);
        out[((int64_t)z * my + y) * mx + x] = (T)U[s * PSLOT + c];
    }
}

// phi and -grad phi (central differences) of the dense root potential into
// the slots; the dense array is [mz][my][mx] and indices wrap modulo those
// extents (the box itself when periodic; the padded grid, whose layers just
// outside the box hold the potential there, when isolated)
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_bits(x); }

template <typename T>  // the transform's precision; differences in FP64
__global__ void k_root_out(const T *__restrict__ phi, const int32_t *__restrict__ corner, int n_patches, int nx,
                           int ny, int nz, double dh, int order, double *__restrict__ phi_out,
                           double *__restrict__ acc_out) {
    const double inv2 = 0.5 / dh, inv12 = 1.0 / (12.0 * dh);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n_patches * PV;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / PV;
        const int c = (int)(i % PV);
        const int x = corner[3 * s] + (c & 7), y = corner[3 * s + 1] + ((c >> 3) & 7),
                  z = corner[3 * s + 2] + (c >> 6);
        auto wrap = [](int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); };  // |offset| <= 2 < n
        auto at = [&](int a, int b, int d) {  // an FP32 value widened exactly on the integer units
            return to_f64(phi[((int64_t)wrap(d, nz) * ny + wrap(b, ny)) * nx + wrap(a, nx)]);
        };
        phi_out[s * PV + c] = at(x, y, z);
        if (!acc_out) continue;
        for (int d = 0; d < 3; d++) {
            const int ex = d == 0, ey = d == 1, ez = d == 2;
            double g;
            if (order == 2) {
                g = (at(x + ex, y + ey, z + ez) - at(x - ex, y - ey, z - ez)) * inv2;
            } else {
                g = (-at(x + 2 * ex, y + 2 * ey, z + 2 * ez) + 8.0 * at(x + ex, y + ey, z + ez) -
                     8.0 * at(x - ex, y - ey, z - ez) + at(x - 2 * ex, y - 2 * ey, z - 2 * ez)) *
                    inv12;
            }
            acc_out[(s * 3 + d) * PV + c] = -g;
        }
    }
}

// ---- refined levels -------------------------------------------------------------

// real: the solve's precision (double, or float in the FP32-compute mode);
// the parent level's potential and the states are read in FP64, the
// potential and accelerations written in FP64
// Rows of the grid padded to 24 values in FP32: the 8 same-colour cells of
// a row sit 2 apart, a warp covers 4 rows, and with a row stride of 24
// words rows j and j+2 (same colour parity) fall on disjoint banks, so a
// sweep's loads are free of bank conflicts (a stride of 18 makes them
// 2-way).  FP64 values take two banks each and keep the dense layout.
template <typename real>
struct SorGeo {
    static constexpr int PX = sizeof(real) == 4 ? 24 : PN;
};

template <typename real>
struct SorSmem {
    real phi[PN][PN][SorGeo<real>::PX];
    real rho[PN][PN][SorGeo<real>::PX];
    int nb[27], cnb[27];  // same-level patches around the patch, parent-level patches around its parent
    int off[3];           // the patch's lower corner relative to its parent's, in coarse cells (0 or 4)
};

template <typename real>
__device__ __forceinline__ real quad1(real pm, real p0, real pp, real x) {
    return p0 + x * (pp - pm) / real(2) + x * x * (pp - real(2) * p0 + pm) / real(2);
}

// a value of a parent-level field at coarse cell c relative to the parent's
// lower corner (each coordinate in -8..15)
__device__ __forceinline__ double coarse_at(const double *__restrict__ F, int64_t stride, const int *cnb, int cx,
                                            int cy, int cz) {
    const int k = ((cx >> 3) + 1) + 3 * ((cy >> 3) + 1) + 9 * ((cz >> 3) + 1);
    return F[(int64_t)cnb[k] * stride + (cz & 7) * 64 + (cy & 7) * 8 + (cx & 7)];
}

// the parent's potential at coarse cell c, linear in time between two
// potentials when F1 is given: (1 - w) F0 + w F1
__device__ __forceinline__ double coarse_phi(const double *__restrict__ F0, const double *__restrict__ F1, double w,
                                             const int *cnb, int cx, int cy, int cz) {
    const double a = coarse_at(F0, PV, cnb, cx, cy, cz);
    if (!F1) return a;
    return (1.0 - w) * a + w * coarse_at(F1, PV, cnb, cx, cy, cz);
}

template <typename real>
__global__ void __launch_bounds__(SOR_NT) k_sor_patches(
    const double *__restrict__ U, const int32_t *__restrict__ sib, const int32_t *__restrict__ parent,
    const int32_t *__restrict__ corner, const double *__restrict__ Uc, const int32_t *__restrict__ csib,
    const int32_t *__restrict__ ccorner, const double *__restrict__ phic, const double *__restrict__ phic1,
    double w, int n_patches, double dh, double G, double omega, int iters, int order, double *__restrict__ phi_out,
    double *__restrict__ acc_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SorSmem<real> &S = *reinterpret_cast<SorSmem<real> *>(smem_raw);
    real *rho_flat = &S.rho[0][0][0], *phi_flat = &S.phi[0][0][0];
    const int tid = threadIdx.x;
    const double src_scale = dh * dh * FOUR_PI * G;
    // phi <- (1 - omega) phi + (omega/6) (sum of the 6 neighbours) - (omega/6) dh^2 4 pi G rho:
    // the same update as phi + omega (sum - 6 phi - dh^2 4 pi G rho) / 6 in
    // five additions and two FMAs, with the source term premultiplied
    const real w6 = (real)(omega / 6.0), om1 = (real)(1.0 - omega);
    const double src_scale_w = -(omega / 6.0) * src_scale;
    const double inv2 = 0.5 / dh, inv12 = 1.0 / (12.0 * dh);
    const real qm = real(-0.25), qp = real(0.25);
    for (int p = blockIdx.x; p < n_patches; p += gridDim.x) {
        if (tid < 27) {
            const int P = parent[p];
            S.nb[tid] = tid == 13 ? p : sib[(int64_t)p * 26 + tid - (tid > 13)];
            const int cs = tid == 13 ? P : csib[(int64_t)P * 26 + tid - (tid > 13)];
            S.cnb[tid] = cs >= 0 ? cs : P;  // present on a properly nested hierarchy
            if (tid < 3) S.off[tid] = corner[3 * p + tid] / 2 - ccorner[3 * P + tid];
        }
        __syncthreads();
        // initial guess on the 18^3 grid: quadratic interpolation along x, then
        // y, then z, each pass once per distinct value (coarse rows -4..7
        // around the patch in y and z: 12 x 12 x 18 along x into the phi
        // array, 12 x 18 x 18 along y into the rho array, then all cells)
        constexpr int NC = 12;
        for (int i = tid; i < NC * NC * PN; i += SOR_NT) {
            const int fx = i % PN, b = (i / PN) % NC, a = i / (PN * NC);
            const int gx = fx - PB, cx = S.off[0] + (gx >> 1);
            const int cy = S.off[1] + b - 4, cz = S.off[2] + a - 4;
            phi_flat[i] = quad1<real>((real)coarse_phi(phic, phic1, w, S.cnb, cx - 1, cy, cz),
                                      (real)coarse_phi(phic, phic1, w, S.cnb, cx, cy, cz),
                                      (real)coarse_phi(phic, phic1, w, S.cnb, cx + 1, cy, cz), (gx & 1) ? qp : qm);
        }
        __syncthreads();
        for (int i = tid; i < NC * PN * PN; i += SOR_NT) {
            const int fx = i % PN, fy = (i / PN) % PN, a = i / (PN * PN);
            const int gy = fy - PB, b = (gy >> 1) + 4;
            const real *X = phi_flat + (a * NC + b) * PN + fx;
            rho_flat[i] = quad1<real>(X[-PN], X[0], X[PN], (gy & 1) ? qp : qm);
        }
        __syncthreads();
        for (int i = tid; i < PN3; i += SOR_NT) {
            const int gz = i / (PN * PN) - PB, a = (gz >> 1) + 4;
            const real *Y = rho_flat + a * PN * PN + i % (PN * PN);
            S.phi[i / (PN * PN)][(i / PN) % PN][i % PN] =
                quad1<real>(Y[-PN * PN], Y[0], Y[PN * PN], (gz & 1) ? qp : qm);
        }
        __syncthreads();
        // the source term -(omega/6) dh^2 4 pi G rho on the grid, formed once per cell
        for (int i = tid; i < PN3; i += SOR_NT) {
            const int gx = i % PN - PB, gy = (i / PN) % PN - PB, gz = i / (PN * PN) - PB;  // fine, relative
            const int k = ((gx >> 3) + 1) + 3 * ((gy >> 3) + 1) + 9 * ((gz >> 3) + 1);
            const int s = S.nb[k];
            S.rho[i / (PN * PN)][(i / PN) % PN][i % PN] =
                (real)(src_scale_w * (s >= 0 ? U[(int64_t)s * PSLOT + (gz & 7) * 64 + (gy & 7) * 8 + (gx & 7)]
                                                      : coarse_at(Uc, PSLOT, S.cnb, S.off[0] + (gx >> 1),
                                                                  S.off[1] + (gy >> 1), S.off[2] + (gz >> 1))));
        }
        __syncthreads();
        // red-black SOR on the interior 16^3 cells
        for (int it = 0; it < iters; it++) {
            for (int colour = 0; colour < 2; colour++) {
                for (int t = tid; t < 2048; t += SOR_NT) {
                    const int row = t >> 3, k = row / 16 + 1, j = row % 16 + 1;
                    const int i = 1 + ((1 + j + k + colour) & 1) + 2 * (t & 7);
                    const real ph = S.phi[k][j][i];
                    const real nbs = S.phi[k - 1][j][i] + S.phi[k + 1][j][i] + S.phi[k][j - 1][i] +
                                     S.phi[k][j + 1][i] + S.phi[k][j][i - 1] + S.phi[k][j][i + 1];
                    S.phi[k][j][i] = fma(w6, nbs, fma(om1, ph, S.rho[k][j][i]));
                }
                __syncthreads();
            }
        }
        // the active cells' potential and acceleration (differences in FP64)
        for (int c = tid; c < PV; c += SOR_NT) {
            const int x = (c & 7) + PB, y = ((c >> 3) & 7) + PB, z = (c >> 6) + PB;
            phi_out[(int64_t)p * PV + c] = (double)S.phi[z][y][x];
            if (!acc_out) continue;
            for (int d = 0; d < 3; d++) {
                const int ex = d == 0, ey = d == 1, ez = d == 2;
                const double p1 = S.phi[z + ez][y + ey][x + ex], m1 = S.phi[z - ez][y - ey][x - ex];
                double g;
                if (order == 2) {
                    g = (p1 - m1) * inv2;
                } else {
                    const double p2 = S.phi[z + 2 * ez][y + 2 * ey][x + 2 * ex],
                                 m2 = S.phi[z - 2 * ez][y - 2 * ey][x - 2 * ex];
                    g = (-p2 + 8.0 * p1 - 8.0 * m1 + m2) * inv12;
                }
                acc_out[((int64_t)p * 3 + d) * PV + c] = -g;
            }
        }
        __syncthreads();
    }
}

// The corrector of the gravity coupling on every cell: momentum from the
// accelerations at both ends of the step, then energy with the corrected
// momentum.  U1: the predicted state (corrected in place), U0: U^n; dt from
// the host or, when negative, the step's device time record.  Fused: the CFL
// signal speed of the corrected state (as the max-speed pass, in the step's
// precision) into smax / n_bad.
template <typename real>
__global__ void k_grav_correct(double *__restrict__ U1, const double *__restrict__ U0,
                               const double *__restrict__ g0, const double *__restrict__ g1, int64_t n_cells,
                               double dt_in, const double *__restrict__ time_rec, double gamma, int cfl1,
                               unsigned long long *smax, unsigned long long *n_bad) {
    const double dt = dt_in >= 0.0 ? dt_in : time_rec[0];
    const double h = 0.5 * dt;
    Gas<real> gas;
    gas.gamma = (real)gamma;
    gas.gm1 = (real)(gamma - 1.0);
    gas.inv_gm1 = (real)(1.0 / (gamma - 1.0));
    double m = 0.0;
    unsigned bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cells;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i / PV;
        const int c = (int)(i % PV);
        const double *u0 = U0 + s * PSLOT + c;
        double *u1 = U1 + s * PSLOT + c;
        double a0[3], a1[3], m1[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            a0[d] = g0[(s * 3 + d) * PV + c];
            a1[d] = g1[(s * 3 + d) * PV + c];
        }
        const double r0 = u0[0], r1 = u1[0];
#pragma unroll
        for (int d = 0; d < 3; d++) m1[d] = u1[(1 + d) * PV] + h * (r0 * a0[d] + r1 * a1[d]);
        const double e0 = u0[PV] * a0[0] + u0[2 * PV] * a0[1] + u0[3 * PV] * a0[2];
        const double e1 = m1[0] * a1[0] + m1[1] * a1[1] + m1[2] * a1[2];
        const double E1 = u1[4 * PV] + h * (e0 + e1);
        u1[4 * PV] = E1;
#pragma unroll
        for (int d = 0; d < 3; d++) u1[(1 + d) * PV] = m1[d];
        real u[NV] = {to_real<real>(r1), to_real<real>(m1[0]), to_real<real>(m1[1]), to_real<real>(m1[2]),
                      to_real<real>(E1)};
        bool ok;
        const real sp = cfl_speed(u, gas, ok, cfl1 != 0);
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

// max over the values of (cfl / c_acc) sqrt(dh |a|): warp maxima, one atomic each
__global__ void k_acc_speed(const double *__restrict__ acc, int64_t n, double dh, double scale,
                            unsigned long long *smax) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(acc[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(smax, (unsigned long long)__double_as_longlong(scale * sqrt(dh * m)));
}

}  // namespace

amr_status launch_acc_speed(amr_hydro_ctx *c, const double *acc, int64_t n_values, double dh, double c_acc,
                            unsigned long long *smax) {
    k_acc_speed<<<c->n_sm * 8, 256, 0, c->stream>>>(acc, n_values, dh, c->prm.cfl / c_acc, smax);
    return cuda_fail(cudaGetLastError(), "k_acc_speed");
}

template <typename real>
amr_status launch_sor(amr_hydro_ctx *c, Level &L, Level &C, int level, double G, double omega, int iters,
                      const double *phi_coarse, const double *phi_coarse1, double w, double *phi, double *acc,
                      int acc_order) {
    static DeviceOnce once;
    amr_status st = once_per_device(once, [] {
        return cuda_fail(cudaFuncSetAttribute(k_sor_patches<real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)sizeof(SorSmem<real>)),
                         "sor smem attribute");
    });
    if (st) return st;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sor_patches<real>, SOR_NT, sizeof(SorSmem<real>));
    const int cap = c->n_sm * (per_sm > 0 ? per_sm : 1);
    const int grid = L.n_patches < cap ? L.n_patches : cap;
    k_sor_patches<real><<<grid, SOR_NT, sizeof(SorSmem<real>), c->stream>>>(
        L.U[L.cur], L.d_sib, L.d_parent, L.d_corner, C.U[C.cur], C.d_sib, C.d_corner, phi_coarse, phi_coarse1, w,
        L.n_patches, level_dh(c, level), G, omega, iters, acc_order, phi, acc);
    return cuda_fail(cudaGetLastError(), "k_sor_patches");
}

// Isolated root potential: the kernel's transform once per context (a full
// forward transform of k_iso_kernel's grid), then per solve the density
// scattered into planes z < nz of the zeroed padded grid and the pruned
// convolution of fft_convolve_isolated (fft.cu): the forward (y, x)
// transforms on those planes only, every (ky, kx) column along z with the
// product by the kernel's transform between its forward and inverse
// transforms, the inverse (y, x) transforms only on the planes the outputs
// read (z < nz + 2 and the two planes below z = 0).  Same arithmetic as the
// full 3-D transform, about 0.6 of its work.
template <typename T>
amr_status root_isolated(amr_hydro_ctx *c, Level &L, int nx, int ny, int nz, int mx, int my, int mz, double G,
                         double *phi, double *acc, int acc_order) {
    (void)nx;
    (void)ny;
    amr_status st;
    const int grid = c->n_sm * 8;
    const int64_t n = (int64_t)mx * my * mz;
    cudaStream_t s = c->stream;
    T *R = reinterpret_cast<T *>(c->fft_real.p);
    const double dh = level_dh(c, 0);
    if (!c->fft_green_ready) {
        k_iso_kernel<T><<<grid, 256, 0, s>>>(R, mx, my, mz, dh);
        if ((st = cuda_fail(cudaGetLastError(), "k_iso_kernel"))) return st;
        if ((st = fft_forward_full<T>(c, R, mx, my, mz, c->fft_green.p, s))) return st;
        c->fft_green_ready = true;
    }
    if ((st = cuda_fail(cudaMemsetAsync(R, 0, sizeof(T) * (int64_t)nz * my * mx, s), "memset padded"))) return st;
    k_rho_scatter<T><<<grid, 256, 0, s>>>(L.U[L.cur], L.d_corner, L.n_patches, mx, my, R);
    if ((st = cuda_fail(cudaGetLastError(), "k_rho_scatter"))) return st;
    if ((st = fft_convolve_isolated<T>(c, R, mx, my, mz, nz, c->fft_green.p, G / (double)n, c->fft_cplx.p, s)))
        return st;
    k_root_out<T><<<grid, 256, 0, s>>>(R, L.d_corner, L.n_patches, mx, my, mz, dh, acc_order, phi, acc);
    return cuda_fail(cudaGetLastError(), "k_root_out");
}

void release_poisson(amr_hydro_ctx *c) {
    c->fft_real.release();
    c->fft_cplx.release();
    c->fft_green.release();
    c->fft_green_ready = false;
    c->fft_tw.release();
    c->fft_tw_n[0] = c->fft_tw_n[1] = c->fft_tw_n[2] = 0;
}

// The gravity corrector of a level just advanced by its predictor (U[cur]
// the predicted state, U[1 - cur] U^n); its fused signal speed replaces the
// step's, which was of the predicted state.
amr_status launch_grav_correct(amr_hydro_ctx *c, int level, double dt, const double *acc_n, const double *acc_new) {
    Level &L = c->lv[level];
    amr_status st;
    unsigned long long *sm = c->scal.p + L.scal0 + L.ring, *nb = c->scal.p + L.scal0 + 3 + L.ring;
    if ((st = cuda_fail(cudaMemsetAsync(sm, 0, 8, c->stream), "memset")) ||
        (st = cuda_fail(cudaMemsetAsync(nb, 0, 8, c->stream), "memset")))
        return st;
    const int64_t n_cells = (int64_t)L.n_patches * PV;
    const int cfl1 = c->prm.scheme == AMR_SCHEME_CTU;  // Eq. (CFL1) for CTU, else Eq. (CFL2)
    const double *rec = c->dtbuf.p + 3 * level;
    if (c->prm.prec == AMR_FP64)
        k_grav_correct<double><<<c->n_sm * 8, 256, 0, c->stream>>>(L.U[L.cur], L.U[1 - L.cur], acc_n, acc_new,
                                                                    n_cells, dt, rec, c->prm.gamma, cfl1, sm, nb);
    else
        k_grav_correct<float><<<c->n_sm * 8, 256, 0, c->stream>>>(L.U[L.cur], L.U[1 - L.cur], acc_n, acc_new,
                                                                   n_cells, dt, rec, c->prm.gamma, cfl1, sm, nb);
    if ((st = cuda_fail(cudaGetLastError(), "k_grav_correct"))) return st;
    L.speed_valid = true;
    L.version++;
    return AMR_OK;
}

}  // namespace amrh

using namespace amrh;

extern "C" {

amr_status amr_hydro_poisson_root(amr_hydro_ctx *c, double G, double *phi, double *acc, int acc_order) {
    if (!c || !phi || (acc && acc_order != 2 && acc_order != 4)) return AMR_E_INVAL;
    Level &L = c->lv[0];
    const int nx = c->prm.root_n[0], ny = c->prm.root_n[1], nz = c->prm.root_n[2];
    if ((int64_t)L.n_patches * PV != (int64_t)nx * ny * nz) return AMR_E_INVAL;  // the whole root grid
    const bool iso = c->prm.gravity_bc == AMR_GRAVITY_ISOLATED;
    // the transformed grid: the box (periodic) or the zero-padded one
    // (isolated; even along x, where the real transforms run)
    const int mx = iso ? smooth7_even(2 * nx + 4) : nx, my = iso ? smooth7(2 * ny + 4) : ny,
              mz = iso ? smooth7(2 * nz + 4) : nz;
    const int64_t n = (int64_t)mx * my * mz, nc = (int64_t)mz * my * (mx / 2 + 1);
    amr_status st;
    // FP64 transforms, or FP32 ones in the FP32-compute mode (potential and
    // accelerations still written in FP64)
    const bool f32 = c->prm.prec != AMR_FP64;
    const int grid = c->n_sm * 8;
    // periodic: the complex spectrum, the per-axis eigenvalue tables, the
    // partial sums of rho; isolated: the spectrum and the kernel's transform
    if ((st = c->fft_real.reserve(n)) || (st = c->fft_cplx.reserve(2 * nc + (iso ? 0 : mx / 2 + 1 + my + mz + grid))) ||
        (iso && (st = c->fft_green.reserve(2 * nc))))
        return st;
    if (iso)
        return f32 ? root_isolated<float>(c, L, nx, ny, nz, mx, my, mz, G, phi, acc, acc_order)
                   : root_isolated<double>(c, L, nx, ny, nz, mx, my, mz, G, phi, acc, acc_order);
    cudaStream_t s = c->stream;
    const double dh = level_dh(c, 0);
    double *lam1 = c->fft_cplx.p + 2 * nc, *partial = lam1 + nx / 2 + 1 + ny + nz;
    k_rho_partial<<<grid, 256, 0, s>>>(L.U[L.cur], L.n_patches, partial);
    if ((st = cuda_fail(cudaGetLastError(), "k_rho_partial"))) return st;
    k_green_axes<<<(nx / 2 + 1 + ny + nz + 255) / 256, 256, 0, s>>>(lam1, nx, ny, nz);
    if ((st = cuda_fail(cudaGetLastError(), "k_green_axes"))) return st;
    const double scale = FOUR_PI * G * dh * dh / (double)n;
    // our transforms (fft.cu): the real field in place, the half spectrum in
    // fft_cplx, the Green's factor applied between the z transforms
    if (f32) {
        float *R = reinterpret_cast<float *>(c->fft_real.p);
        k_rho_dense<float><<<grid, 256, 0, s>>>(L.U[L.cur], L.d_corner, L.n_patches, nx, ny, partial, grid, R);
        if ((st = cuda_fail(cudaGetLastError(), "k_rho_dense"))) return st;
        if ((st = fft_poisson_periodic<float>(c, R, nx, ny, nz, lam1, scale, c->fft_cplx.p, s))) return st;
        k_root_out<float><<<grid, 256, 0, s>>>(R, L.d_corner, L.n_patches, nx, ny, nz, dh, acc_order, phi, acc);
    } else {
        double *R = c->fft_real.p;
        k_rho_dense<double><<<grid, 256, 0, s>>>(L.U[L.cur], L.d_corner, L.n_patches, nx, ny, partial, grid, R);
        if ((st = cuda_fail(cudaGetLastError(), "k_rho_dense"))) return st;
        if ((st = fft_poisson_periodic<double>(c, R, nx, ny, nz, lam1, scale, c->fft_cplx.p, s))) return st;
        k_root_out<double><<<grid, 256, 0, s>>>(R, L.d_corner, L.n_patches, nx, ny, nz, dh, acc_order, phi, acc);
    }
    return cuda_fail(cudaGetLastError(), "k_root_out");
}

amr_status amr_hydro_advance_gravity(amr_hydro_ctx *c, double dt, double G, const double *acc_n, double *phi_new,
                                     double *acc_new, int acc_order, double c_acc) {
    if (!c || !acc_n || !phi_new || !acc_new || (acc_order != 2 && acc_order != 4)) return AMR_E_INVAL;
    if (!(c_acc >= 0.0) || c_acc > 1e300) return AMR_E_INVAL;
    {  // the corrector reads g^n and the state after the root solve has written
       // phi^{n+1} and g^{n+1}: none of the outputs may overlap g^n, each other
       // or the level's two state buffers
        const Level &L0 = c->lv[0];
        const int64_t nf = (int64_t)L0.n_patches * PV, nu = (int64_t)L0.n_patches * PSLOT;
        if (overlaps(acc_n, 3 * nf, acc_new, 3 * nf) || overlaps(acc_n, 3 * nf, phi_new, nf) ||
            overlaps(phi_new, nf, acc_new, 3 * nf))
            return AMR_E_INVAL;
        for (int b = 0; b < 2; b++)
            if (overlaps(L0.U[b], nu, phi_new, nf) || overlaps(L0.U[b], nu, acc_new, 3 * nf) ||
                overlaps(L0.U[b], nu, acc_n, 3 * nf))
                return AMR_E_INVAL;
    }
    if (!(dt >= 0.0) && !(dt < 0.0)) return AMR_E_INVAL;
    if (c->prm.lmax > 0 && c->lv[1].n_patches) return AMR_E_INVAL;  // single-level grids
    if ((c->prm.scheme != AMR_SCHEME_MH && c->prm.scheme != AMR_SCHEME_CTU) || c->prm.recon != AMR_RECON_PLM ||
        c->prm.dual_energy || c->prm.fallback || c->prm.dt_min > 0.0)
        return AMR_E_INVAL;
    Level &L = c->lv[0];
    if (!L.n_patches || L.n_ghost) return AMR_E_INVAL;
    amr_status st;
    // predictor: the hydro step with gravity in the half step
    if ((st = advance_once(c, 0, dt, nullptr, acc_n, c_acc))) return st;
    // the potential and acceleration of the predicted density
    if ((st = amr_hydro_poisson_root(c, G, phi_new, acc_new, acc_order))) return st;
    // corrector (the step flipped the buffers: U[cur] is the predicted state)
    return launch_grav_correct(c, 0, dt, acc_n, acc_new);
}

static amr_status poisson_level(amr_hydro_ctx *c, int level, double G, double omega, int iters,
                                const double *phi_c0, const double *phi_c1, double w, double *phi, double *acc,
                                int acc_order) {
    if (!c || level < 1 || level > c->prm.lmax || !phi_c0 || !phi || iters < 0) return AMR_E_INVAL;
    if (acc && acc_order != 2 && acc_order != 4) return AMR_E_INVAL;
    if (!(w >= 0.0 && w <= 1.0)) return AMR_E_INVAL;
    Level &L = c->lv[level], &C = c->lv[level - 1];
    if (!L.n_patches) return AMR_OK;
    if (!L.d_parent || !C.n_patches) return AMR_E_INVAL;
    // the outputs are written while other CTAs still read the parent's potential
    const int64_t nf = (int64_t)L.n_patches * PV, ncp = (int64_t)C.n_patches * PV;
    if (overlaps(phi, nf, phi_c0, ncp) || overlaps(phi, nf, phi_c1, ncp) || overlaps(acc, 3 * nf, phi_c0, ncp) ||
        overlaps(acc, 3 * nf, phi_c1, ncp) || overlaps(phi, nf, acc, 3 * nf))
        return AMR_E_INVAL;
    // FP64, or FP32 in the FP32-compute mode (half the shared memory: 4 CTAs per SM)
    return c->prm.prec == AMR_FP64
               ? launch_sor<double>(c, L, C, level, G, omega, iters, phi_c0, phi_c1, w, phi, acc, acc_order)
               : launch_sor<float>(c, L, C, level, G, omega, iters, phi_c0, phi_c1, w, phi, acc, acc_order);
}

amr_status amr_hydro_poisson_level(amr_hydro_ctx *c, int level, double G, double omega, int iters,
                                   const double *phi_coarse, double *phi, double *acc, int acc_order) {
    return poisson_level(c, level, G, omega, iters, phi_coarse, nullptr, 0.0, phi, acc, acc_order);
}

amr_status amr_hydro_poisson_level_t(amr_hydro_ctx *c, int level, double G, double omega, int iters,
                                     const double *phi_coarse_old, const double *phi_coarse_new, double w,
                                     double *phi, double *acc, int acc_order) {
    if (!phi_coarse_new) return AMR_E_INVAL;
    return poisson_level(c, level, G, omega, iters, phi_coarse_old, phi_coarse_new, w, phi, acc, acc_order);
}

}  // extern "C"
