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
}  // namespace

// x: device double[n]; out: device double[10n].
extern "C" int amrh_selftest_math(const double *x, int n, double *out) {
    if (!x || !out || n <= 0) return 1;
    k_selftest_math<<<(n + 255) / 256, 256>>>(x, n, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
