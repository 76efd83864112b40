// noalloc.cu -- one step of a uniform periodic grid that allocates nothing.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// reserved up front by their own pool allocator (another framework's caching
// allocator already holds the memory, so a late cudaMalloc may fail or
// fragment it), and latency-critical loops that cannot take the implicit
// device-wide synchronisation cudaMalloc/cudaFree may cause.  Creating a
// context (amr_hydro_init / amr_hydro_set_level) allocates its scratch, so
// this entry point runs the same fused step kernel with its scratch -- the
// per-group neighbour table and the reduction scalars -- in a file-scope
// static device array instead.  The caller passes inputs and outputs.
//
// The array is NOALLOC_MAX_GROUPS * 64 int32 plus 8 uint64 (1 MiB + 64 B)
// and every GPU that loads this library holds it until the process exits.
// All calls share it and it keeps the last call's contents: each call
// rebuilds the neighbour table and zeroes the scalars it accumulates into,
// and calls that overlap on the GPU (different streams, or host threads)
// race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "amr_hydro.h"
#include "ctx.h"
#include "step_kernel.cuh"

using namespace amrh;

namespace {

constexpr int NOALLOC_MAX_GROUPS = AMR_NOALLOC_MAX_GROUPS;
constexpr int NOALLOC_SCALARS = 8;  // uint64 words before the table
constexpr size_t NOALLOC_WORDS = NOALLOC_SCALARS + (size_t)NOALLOC_MAX_GROUPS * 64 / 2;

static __device__ __align__(256) unsigned long long noalloc_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex setup_mutex;
void *scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (in host code the symbol itself is only a host-side stand-in).
amr_status scratch_for_current_device(void **out) {
    int dev = 0;
    amr_status st = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
    if (st) return st;
    if (dev < 0 || dev >= MAX_DEVICES) return AMR_E_INVAL;
    std::lock_guard<std::mutex> lock(setup_mutex);
    if (!scratch_addr[dev]) {
        void *p = nullptr;
        if ((st = cuda_fail(cudaGetSymbolAddress(&p, noalloc_scratch), "cudaGetSymbolAddress"))) return st;
        scratch_addr[dev] = p;
    }
    *out = scratch_addr[dev];
    return AMR_OK;
}

// Neighbour table of a fully covered periodic level in the uniform slot order
// (group g = gx + ngx (gy + ngy gz), slot = 8 g + px + 2 py + 4 pz).
__global__ void k_uniform_nbr(int32_t *nbr, int ngx, int ngy, int ngz) {
    const int64_t total = (int64_t)ngx * ngy * ngz * 64;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = (int)(i & 63);
        const int64_t g = i >> 6;
        const int gx = (int)(g % ngx), gy = (int)((g / ngx) % ngy), gz = (int)(g / ((int64_t)ngx * ngy));
        const int qx = (pos & 3) - 1, qy = ((pos >> 2) & 3) - 1, qz = (pos >> 4) - 1;
        const int npx = 2 * ngx, npy = 2 * ngy, npz = 2 * ngz;
        const int px = (2 * gx + qx + npx) % npx, py = (2 * gy + qy + npy) % npy, pz = (2 * gz + qz + npz) % npz;
        const int64_t gg = (px >> 1) + (int64_t)ngx * ((py >> 1) + (int64_t)ngy * (pz >> 1));
        nbr[i] = (int32_t)(8 * gg + (px & 1) + 2 * (py & 1) + 4 * (pz & 1));
    }
}

__global__ void k_noalloc_outputs(const unsigned long long *scal, double cfl, double dh, double *dt_next,
                                  unsigned long long *n_bad) {
    const double s = __longlong_as_double((long long)scal[1]);
    const unsigned long long nb = scal[4];
    if (dt_next) *dt_next = (nb || !(s > 0.0)) ? -1.0 : cfl * dh / s;
    if (n_bad) *n_bad = nb;
}

}  // namespace

extern "C" amr_status amr_hydro_step_uniform_noalloc(const double *U_old, double *U_new, int nx, int ny,
                                                     int nz, double dh, double dt, double gamma, double cfl,
                                                     int prec, double *dt_next_out,
                                                     unsigned long long *n_unphysical_out,
                                                     void *cuda_stream) {
    if (!U_old || !U_new || U_old == U_new) return AMR_E_INVAL;
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx % 16 || ny % 16 || nz % 16) return AMR_E_INVAL;
    if (!(dh > 0.0) || !(dt >= 0.0) || !std::isfinite(dt) || !(gamma > 1.0) || !(cfl > 0.0)) return AMR_E_INVAL;
    if (prec != AMR_FP64 && prec != AMR_FP32_ACC64) return AMR_E_INVAL;
    const int64_t n_groups = (int64_t)(nx / 16) * (ny / 16) * (nz / 16);
    if (n_groups > NOALLOC_MAX_GROUPS) {
        std::fprintf(stderr,
                     "amr_hydro_step_uniform_noalloc: %lld patch groups (%dx%dx%d cells) exceed the static "
                     "scratch limit of %d groups (e.g. 256^3 cells)\n",
                     (long long)n_groups, nx, ny, nz, NOALLOC_MAX_GROUPS);
        return AMR_E_INVAL;
    }
    void *base = nullptr;
    amr_status st = scratch_for_current_device(&base);
    if (st) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned long long *scal = (unsigned long long *)base;
    int32_t *nbr = (int32_t *)(scal + NOALLOC_SCALARS);
    if ((st = cuda_fail(cudaMemsetAsync(scal, 0, sizeof(unsigned long long) * NOALLOC_SCALARS, stream),
                        "memset scratch")))
        return st;
    k_uniform_nbr<<<256, 256, 0, stream>>>(nbr, nx / 16, ny / 16, nz / 16);
    if ((st = cuda_fail(cudaGetLastError(), "k_uniform_nbr"))) return st;

    StepParams P;
    std::memset(&P, 0, sizeof(P));
    P.U_old = U_old;
    P.U_new = U_new;
    P.nbr = nbr;
    P.n_work = (int)n_groups;
    P.dt = dt;
    P.cfl = cfl;
    P.dh = dh;
    P.gamma = gamma;
    P.smax_in = scal + 0;
    P.smax_out = scal + 1;
    P.clear2 = scal + 2;  // zeroes scal[2] and scal[5], which nothing reads
    P.n_bad = scal + 4;
    if ((st = launch_step_raw(prec, P, stream))) return st;
    if (dt_next_out || n_unphysical_out) {
        k_noalloc_outputs<<<1, 1, 0, stream>>>(scal, cfl, dh, dt_next_out, n_unphysical_out);
        if ((st = cuda_fail(cudaGetLastError(), "k_noalloc_outputs"))) return st;
    }
    return AMR_OK;
}
