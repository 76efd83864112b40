// fft.h -- the root level's Poisson solves (periodic, and the isolated
// zero-padded convolution) with our own transforms (fft.cu).
#pragma once
#include <cuda_runtime.h>

#include "amr_hydro.h"

struct amr_hydro_ctx;

namespace amrh {

// One transform axis: its length and the radices of its Stockham stages.
struct FftAxis {
    int n = 0;
    int nrad = 0;
    int rad[24] = {};
};

// Radix sequence of a length (4s first, then 2, 3, 5, 7, other primes);
// false when a prime factor exceeds the direct-DFT stage's limit (64).
bool fft_factor(int n, FftAxis &ax);

// phi = FFT^-1[ scale rho_k / lambda_k ] of the dense real field R
// [nz][ny][nx] (in place; the (0,0,0) mode set to zero), lambda_k the
// second-order Laplacian's eigenvalues from the per-axis table lam1 (x: nx/2+1
// entries, then y, then z).  T: double, or float in the FP32-compute mode.
// spec: the half spectrum's storage, nz ny (nx/2+1) complex values of T.
template <typename T>
amr_status fft_poisson_periodic(amr_hydro_ctx *c, T *R, int nx, int ny, int nz, const double *lam1, double scale,
                                void *spec, cudaStream_t s);

// The forward transform of the real field R [mz][my][mx] (mx even) into its
// half spectrum spec [mz][my][mx/2+1] (R is overwritten by nothing).
template <typename T>
amr_status fft_forward_full(amr_hydro_ctx *c, T *R, int mx, int my, int mz, void *spec, cudaStream_t s);

// The zero-padded convolution of the isolated root solve: R [mz][my][mx]
// holds data on planes z < nz (zero elsewhere; those planes are not read);
// R <- FFT^-1[ scale FFT[R] gk ] (gk: a half spectrum as fft_forward_full
// makes, the product formed in FP64), written on the planes z < nz + 2 and
// z >= mz - 2 only (the ones the potential's differences read).  The
// transforms are pruned to those planes; the arithmetic is the full 3-D
// transform's.  spec: the half spectrum's storage.
template <typename T>
amr_status fft_convolve_isolated(amr_hydro_ctx *c, T *R, int mx, int my, int mz, int nz, const void *gk,
                                 double scale, void *spec, cudaStream_t s);

}  // namespace amrh
