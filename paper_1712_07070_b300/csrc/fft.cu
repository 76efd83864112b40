// fft.cu -- our own discrete Fourier transforms for the root level's periodic
// Poisson solve (GAMER-2 section 2.3: the density convolved with the Green's
// function of the second-order Laplacian in Fourier space).
//
// The 3-D transform runs axis by axis on the GPU, each pass a batch of 1-D
// transforms held in shared memory:
//   x  (forward)   two real rows packed as one complex row, one complex
//                  transform, then separated into the two half spectra
//                  (the real input's Hermitian symmetry: nx/2 + 1 columns);
//   y  (forward)   complex columns, tiles of consecutive k_x (coalesced);
//   z  (forward, the Green's factor, inverse) in one pass per column tile;
//   y  (inverse);
//   x  (inverse)   two half spectra combined as A + iB, one complex inverse,
//                  the real and imaginary parts are the two rows.
// Each 1-D transform is a mixed-radix Stockham autosort FFT (Stockham 1966;
// the GPU formulation of Govindaraju et al. 2008): stages of radix 4, 2, 3,
// 5, 7 (and a direct DFT stage for any other prime factor), twiddles from a
// per-axis table of exp(-2 pi i t / n) computed with sincospi.  The inverse
// transforms are unnormalised; the 1/N goes into the Green's factor.
#include <cuda_runtime.h>

#include "amr_hydro.h"
#include "ctx.h"
#include "fft.h"

namespace amrh {

template <typename T>
struct Cx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) {
    return {a.x - b.x, a.y - b.y};
}
// exp(sign 2 pi i t / n) from the table of exp(-2 pi i t / n)
template <typename T>
__device__ __forceinline__ Cx<T> twid(const double2 *tw, int t, int sign) {
    const double2 w = tw[t];
    return {(T)w.x, (T)(sign < 0 ? w.y : -w.y)};
}

// Stockham stages over `lines` lines of length ax.n in shared memory: line l
// at a + l * ls, scratch b alike.  Returns the buffer holding the result.
// Every thread of the block takes part (barriers between stages).
template <typename T>
__device__ Cx<T> *fft_smem(Cx<T> *a, Cx<T> *b, int ls, int lines, const FftAxis &ax, const double2 *tw, int sign) {
    const int n = ax.n;
    int Ns = 1;
    for (int st = 0; st < ax.nrad; st++) {
        const int R = ax.rad[st], m = n / R, tscale = n / (Ns * R);
        for (int it = threadIdx.x; it < lines * m; it += blockDim.x) {
            const int l = it / m, j = it - l * m;
            const Cx<T> *in = a + l * ls;
            Cx<T> *out = b + l * ls;
            const int k = j % Ns;
            const int o = (j - k) * R + k;  // (j / Ns) Ns R + j mod Ns
            if (R == 4) {
                Cx<T> v[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    v[r] = in[j + r * m];
                    if (r) v[r] = cmul(v[r], twid<T>(tw, (r * k * tscale) % n, sign));
                }
                const Cx<T> a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), a2 = cadd(v[1], v[3]);
                const Cx<T> d = csub(v[1], v[3]);
                // (v1 - v3) times sign * i
                const Cx<T> a3 = sign < 0 ? Cx<T>{d.y, -d.x} : Cx<T>{-d.y, d.x};
                out[o] = cadd(a0, a2);
                out[o + Ns] = cadd(a1, a3);
                out[o + 2 * Ns] = csub(a0, a2);
                out[o + 3 * Ns] = csub(a1, a3);
            } else if (R == 2) {
                const Cx<T> v0 = in[j], v1 = cmul(in[j + m], twid<T>(tw, (k * tscale) % n, sign));
                out[o] = cadd(v0, v1);
                out[o + Ns] = csub(v0, v1);
            } else {  // a direct DFT of radix R (3, 5, 7 or another prime)
                constexpr int RMAX = 64;
                Cx<T> v[RMAX];
                for (int r = 0; r < R; r++) {
                    v[r] = in[j + r * m];
                    if (r) v[r] = cmul(v[r], twid<T>(tw, (int)(((long long)r * k * tscale) % n), sign));
                }
                for (int p = 0; p < R; p++) {
                    Cx<T> s = v[0];
                    for (int q = 1; q < R; q++) s = cadd(s, cmul(v[q], twid<T>(tw, ((p * q) % R) * m, sign)));
                    out[o + p * Ns] = s;
                }
            }
        }
        __syncthreads();
        Cx<T> *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

}  // namespace amrh

namespace amrh {
namespace {

// tw[t] = exp(-2 pi i t / n), t < n
__global__ void k_twiddles(double2 *tw, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)n, &s, &c);
        tw[t] = make_double2(c, s);
    }
}

// x forward: rows (z, 2p) and (z, 2p + 1) of the real field, packed as one
// complex row (pair p = z ny/2 + y/2 holds rows 2p, 2p + 1), transformed and
// separated into their half spectra A_k = (Z_k + conj Z_{-k}) / 2,
// B_k = (Z_k - conj Z_{-k}) / 2i, k = 0 .. nx/2.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_fwd(const T *__restrict__ R, Cx<T> *__restrict__ S, FftAxis ax,
                                                   const double2 *__restrict__ tw, int64_t n_pairs, int ppb) {
    extern __shared__ __align__(16) unsigned char smem_fft[];
    const int nx = ax.n, nxh = nx / 2 + 1;
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_fft), *b = a + ppb * nx;
    for (int64_t p0 = (int64_t)blockIdx.x * ppb; p0 < n_pairs; p0 += (int64_t)gridDim.x * ppb) {
        const int np = (int)min((int64_t)ppb, n_pairs - p0);
        for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
            const int l = i / nx, x = i - l * nx;
            const int64_t row = 2 * (p0 + l);
            a[l * nx + x] = Cx<T>{R[row * nx + x], R[(row + 1) * nx + x]};
        }
        __syncthreads();
        const Cx<T> *r = fft_smem(a, b, nx, np, ax, tw, -1);
        for (int i = threadIdx.x; i < np * nxh; i += blockDim.x) {
            const int l = i / nxh, k = i - l * nxh;
            const Cx<T> z = r[l * nx + k], w = r[l * nx + (k ? nx - k : 0)];
            const int64_t row = 2 * (p0 + l);
            S[row * nxh + k] = Cx<T>{(z.x + w.x) * T(0.5), (z.y - w.y) * T(0.5)};
            S[(row + 1) * nxh + k] = Cx<T>{(z.y + w.y) * T(0.5), (w.x - z.x) * T(0.5)};
        }
        __syncthreads();
    }
}

// x inverse: the half spectra of rows 2p and 2p + 1 combined as Z = A + iB
// (full length by Hermitian symmetry), one inverse transform; its real and
// imaginary parts are the two rows (unnormalised).
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_inv(const Cx<T> *__restrict__ S, T *__restrict__ R, FftAxis ax,
                                                   const double2 *__restrict__ tw, int64_t n_pairs, int ppb) {
    extern __shared__ __align__(16) unsigned char smem_fft[];
    const int nx = ax.n, nxh = nx / 2 + 1;
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_fft), *b = a + ppb * nx;
    for (int64_t p0 = (int64_t)blockIdx.x * ppb; p0 < n_pairs; p0 += (int64_t)gridDim.x * ppb) {
        const int np = (int)min((int64_t)ppb, n_pairs - p0);
        for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
            const int l = i / nx, k = i - l * nx;
            const int64_t row = 2 * (p0 + l);
            Cx<T> A, B;
            if (k < nxh) {
                A = S[row * nxh + k];
                B = S[(row + 1) * nxh + k];
            } else {  // conjugates of the mirrored columns
                A = S[row * nxh + (nx - k)];
                B = S[(row + 1) * nxh + (nx - k)];
                A.y = -A.y;
                B.y = -B.y;
            }
            a[l * nx + k] = Cx<T>{A.x - B.y, A.y + B.x};
        }
        __syncthreads();
        const Cx<T> *r = fft_smem(a, b, nx, np, ax, tw, +1);
        for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
            const int l = i / nx, x = i - l * nx;
            const int64_t row = 2 * (p0 + l);
            R[row * nx + x] = r[l * nx + x].x;
            R[(row + 1) * nx + x] = r[l * nx + x].y;
        }
        __syncthreads();
    }
}

// Column transforms of the spectrum S [nz][ny][nxh] along y (axis 1) or z
// (axis 2), in tiles of tw_w consecutive k_x of one line position (z for y
// columns, y for z columns), coalesced along k_x.  green (z only): forward,
// times scale / lambda_k (the (0,0,0) mode zeroed), then inverse.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_col(Cx<T> *__restrict__ S, FftAxis ax, const double2 *__restrict__ tw,
                                                 int axis, int nxh, int ny, int nz, int tw_w, int sign, int green,
                                                 const double *__restrict__ lam1, double scale) {
    extern __shared__ __align__(16) unsigned char smem_fft[];
    const int n = ax.n;
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_fft), *b = a + tw_w * n;
    const int ntile = (nxh + tw_w - 1) / tw_w;
    const int other = axis == 1 ? nz : ny;
    const int64_t n_items = (int64_t)other * ntile;
    const int64_t es = axis == 1 ? nxh : (int64_t)ny * nxh;  // stride between a line's elements
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int o = (int)(it / ntile), t = (int)(it - (int64_t)o * ntile);
        const int kx0 = t * tw_w, w_n = min(tw_w, nxh - kx0);
        const int64_t base = axis == 1 ? (int64_t)o * ny * nxh + kx0 : (int64_t)o * nxh + kx0;
        for (int i = threadIdx.x; i < n * tw_w; i += blockDim.x) {
            const int e = i / tw_w, q = i - e * tw_w;
            a[q * n + e] = q < w_n ? S[base + e * es + q] : Cx<T>{T(0), T(0)};
        }
        __syncthreads();
        Cx<T> *r = fft_smem(a, b, n, tw_w, ax, tw, green ? -1 : sign);
        if (green) {  // element e = k_z of column (k_y = o, k_x = kx0 + q)
            for (int i = threadIdx.x; i < n * tw_w; i += blockDim.x) {
                const int q = i / n, e = i - q * n, kx = kx0 + q;
                if (q >= w_n) continue;
                Cx<T> v = r[q * n + e];
                if (kx == 0 && o == 0 && e == 0) {
                    v = Cx<T>{T(0), T(0)};
                } else {
                    const double lam = lam1[kx] + lam1[nxh + o] + lam1[nxh + ny + e];
                    T f;
                    if constexpr (sizeof(T) == sizeof(float)) f = (float)scale / (float)lam;
                    else f = scale / lam;
                    v.x *= f;
                    v.y *= f;
                }
                r[q * n + e] = v;
            }
            __syncthreads();
            r = fft_smem(r, r == a ? b : a, n, tw_w, ax, tw, +1);
        }
        for (int i = threadIdx.x; i < n * tw_w; i += blockDim.x) {
            const int e = i / tw_w, q = i - e * tw_w;
            if (q < w_n) S[base + e * es + q] = r[q * n + e];
        }
        __syncthreads();
    }
}

amr_status set_smem(const void *fn) {
    return cuda_fail(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                     "fft smem attribute");
}

}  // namespace

bool fft_factor(int n, FftAxis &ax) {
    ax.n = n;
    ax.nrad = 0;
    if (n < 1) return false;
    int m = n;
    // radix 4 while a factor 4 remains (the last factor 2 as radix 2)
    while (m % 4 == 0 && ax.nrad < 24) {
        ax.rad[ax.nrad++] = 4;
        m /= 4;
    }
    for (int p = 2; m > 1 && ax.nrad < 24;) {
        if (m % p == 0) {
            if (p > 64) return false;
            ax.rad[ax.nrad++] = p;
            m /= p;
        } else {
            p++;
        }
    }
    return m == 1;
}

template <typename T>
amr_status fft_poisson_periodic(amr_hydro_ctx *c, T *R, int nx, int ny, int nz, const double *lam1, double scale,
                                void *spec, double2 *tw_unused, cudaStream_t s) {
    (void)tw_unused;
    if (nx % 2 || ny % 2) return AMR_E_INVAL;
    FftAxis ax, ay, az;
    if (!fft_factor(nx, ax) || !fft_factor(ny, ay) || !fft_factor(nz, az)) return AMR_E_INVAL;
    amr_status st;
    // per-axis twiddle tables, made once per size
    if (c->fft_tw_n[0] != nx || c->fft_tw_n[1] != ny || c->fft_tw_n[2] != nz) {
        if ((st = c->fft_tw.reserve(2 * (size_t)(nx + ny + nz)))) return st;
        double2 *t = reinterpret_cast<double2 *>(c->fft_tw.p);
        k_twiddles<<<(nx + 255) / 256, 256, 0, s>>>(t, nx);
        k_twiddles<<<(ny + 255) / 256, 256, 0, s>>>(t + nx, ny);
        k_twiddles<<<(nz + 255) / 256, 256, 0, s>>>(t + nx + ny, nz);
        if ((st = cuda_fail(cudaGetLastError(), "k_twiddles"))) return st;
        c->fft_tw_n[0] = nx;
        c->fft_tw_n[1] = ny;
        c->fft_tw_n[2] = nz;
    }
    const double2 *twx = reinterpret_cast<const double2 *>(c->fft_tw.p), *twy = twx + nx, *twz = twy + ny;
    static DeviceOnce once;
    if ((st = once_per_device(once, [] {
             amr_status e;
             if ((e = set_smem((const void *)k_fft_x_fwd<double>)) || (e = set_smem((const void *)k_fft_x_inv<double>)) ||
                 (e = set_smem((const void *)k_fft_col<double>)) || (e = set_smem((const void *)k_fft_x_fwd<float>)) ||
                 (e = set_smem((const void *)k_fft_x_inv<float>)) || (e = set_smem((const void *)k_fft_col<float>)))
                 return e;
             return AMR_OK;
         })))
        return st;
    Cx<T> *S = reinterpret_cast<Cx<T> *>(spec);
    const int nxh = nx / 2 + 1;
    const int64_t n_pairs = (int64_t)nz * ny / 2;
    const int ppb = nx >= 1024 ? 1 : 1024 / nx;
    const size_t sx = 2 * (size_t)ppb * nx * sizeof(Cx<T>);
    const int grid = c->n_sm * 4;
    auto col_w = [](int n) {
        int w = 2048 / n;
        return w < 1 ? 1 : (w > 16 ? 16 : w);
    };
    const int wy = col_w(ny), wz = col_w(nz);
    k_fft_x_fwd<T><<<grid, 256, sx, s>>>(R, S, ax, twx, n_pairs, ppb);
    if ((st = cuda_fail(cudaGetLastError(), "k_fft_x_fwd"))) return st;
    k_fft_col<T><<<grid, 256, 2 * (size_t)wy * ny * sizeof(Cx<T>), s>>>(S, ay, twy, 1, nxh, ny, nz, wy, -1, 0, lam1,
                                                                        scale);
    if ((st = cuda_fail(cudaGetLastError(), "k_fft_col y"))) return st;
    k_fft_col<T><<<grid, 256, 2 * (size_t)wz * nz * sizeof(Cx<T>), s>>>(S, az, twz, 2, nxh, ny, nz, wz, -1, 1, lam1,
                                                                        scale);
    if ((st = cuda_fail(cudaGetLastError(), "k_fft_col z"))) return st;
    k_fft_col<T><<<grid, 256, 2 * (size_t)wy * ny * sizeof(Cx<T>), s>>>(S, ay, twy, 1, nxh, ny, nz, wy, +1, 0, lam1,
                                                                        scale);
    if ((st = cuda_fail(cudaGetLastError(), "k_fft_col y inverse"))) return st;
    k_fft_x_inv<T><<<grid, 256, sx, s>>>(S, R, ax, twx, n_pairs, ppb);
    return cuda_fail(cudaGetLastError(), "k_fft_x_inv");
}

template amr_status fft_poisson_periodic<double>(amr_hydro_ctx *, double *, int, int, int, const double *, double,
                                                 void *, double2 *, cudaStream_t);
template amr_status fft_poisson_periodic<float>(amr_hydro_ctx *, float *, int, int, int, const double *, double,
                                                void *, double2 *, cudaStream_t);

}  // namespace amrh
