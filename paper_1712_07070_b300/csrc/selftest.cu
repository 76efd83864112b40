// selftest.cu -- test hook (not part of the C ABI): evaluates the step
// kernel's own reciprocal / reciprocal-square-root / square-root refinements and the
// integer double<->float conversions next to CUDA's IEEE operations, so the
// tests can bound their error.
#include <cuda_runtime.h>

#include "hydro_math.cuh"

namespace {
__global__ void k_selftest_math(const double *x, int n, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = x[i];
        double *o = out + 10 * (size_t)i;
        o[0] = amrh::rcp_(v);
        o[1] = 1.0 / v;
        o[2] = amrh::rsqrt_(v);
        o[3] = 1.0 / sqrt(v);
        o[4] = (double)amrh::d2f_bits(v);
        o[5] = (double)__double2float_rn(v);
        const float f = __double2float_rn(v);
        o[6] = amrh::f2d_bits(f);
        o[7] = (double)f;
        o[8] = amrh::sqrt_(v);
        o[9] = sqrt(v);
    }
}
// Integer-unit sign tests and min/max next to the FP64 comparisons: bit 0..2
// gt0/ge0/le0 agree, bit 3/4 min_/max_ return the same value (compared as
// numbers, so +0 and -0 count as equal).
__global__ void k_selftest_order(const double *a, const double *b, int n, int *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = a[i], y = b[i];
        int r = 0;
        r |= (amrh::gt0(x) == (x > 0.0)) << 0;
        r |= (amrh::ge0(x) == (x >= 0.0)) << 1;
        r |= (amrh::le0(x) == (x <= 0.0)) << 2;
        r |= (amrh::min_(x, y) == ((x <= y) ? x : y)) << 3;
        r |= (amrh::max_(x, y) == ((x >= y) ? x : y)) << 4;
        out[i] = r;
    }
}
}  // namespace

// x: device double[n]; out: device double[10n].
extern "C" int amrh_selftest_math(const double *x, int n, double *out) {
    if (!x || !out || n <= 0) return 1;
    k_selftest_math<<<(n + 255) / 256, 256>>>(x, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// a, b: device double[n] (no NaNs); out: device int[n], 31 where all agree.
extern "C" int amrh_selftest_order(const double *a, const double *b, int n, int *out) {
    if (!a || !b || !out || n <= 0) return 1;
    k_selftest_order<<<(n + 255) / 256, 256>>>(a, b, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
