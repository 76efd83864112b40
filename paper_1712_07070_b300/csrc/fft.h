// fft.h -- the root level's periodic Poisson solve with our own transforms
// (fft.cu).
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
// Work arrays: spec (nz ny (nx/2+1) complex), tw (the twiddle tables).
template <typename T>
amr_status fft_poisson_periodic(amr_hydro_ctx *c, T *R, int nx, int ny, int nz, const double *lam1, double scale,
                                void *spec, double2 *tw, cudaStream_t s);

}  // namespace amrh
