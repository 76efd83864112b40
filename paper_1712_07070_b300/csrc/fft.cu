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
// 5, 7 (and a paired direct DFT stage for any other odd prime up to 64),
// twiddles from a per-axis table of exp(-2 pi i t / n) computed with
// sincospi (an FP32 copy for the FP32-compute mode).  The inverse
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
// exp(sign 2 pi i t / n) from the table of exp(-2 pi i t / n) (0 <= t < n),
// held in the compute type
template <typename T>
__device__ __forceinline__ Cx<T> twid(const Cx<T> *tw, int t, int sign) {
    const Cx<T> w = tw[t];
    return {w.x, sign < 0 ? w.y : -w.y};
}

// One odd-radix butterfly of radix R: inputs j + q m (q < R) twiddled by
// exp(sign 2 pi i q kt / n), outputs o + p Ns, as the paired DFT described
// at fft_smem.  RC: R at compile time (3, 5, 7: unrolled, in registers).
template <typename T, int RC>
__device__ __forceinline__ void odd_radix(const Cx<T> *in, Cx<T> *out, int j, int m, int kt, int o, int Ns,
                                          const Cx<T> *tw, int sign) {
    constexpr int R = RC, h = (RC - 1) / 2;
    const Cx<T> v0 = in[j];
    Cx<T> sp[h], sm[h];
    Cx<T> y0 = v0;
#pragma unroll
    for (int q = 1; q <= h; q++) {
        const Cx<T> u = cmul(in[j + q * m], twid<T>(tw, q * kt, sign));
        const Cx<T> w = cmul(in[j + (R - q) * m], twid<T>(tw, (R - q) * kt, sign));
        sp[q - 1] = cadd(u, w);
        sm[q - 1] = csub(u, w);
        y0 = cadd(y0, sp[q - 1]);
    }
    out[o] = y0;
#pragma unroll
    for (int p = 1; p <= h; p++) {
        Cx<T> A = v0, B = {T(0), T(0)};
#pragma unroll
        for (int q = 1; q <= h; q++) {
            const Cx<T> w = tw[((p * q) % R) * m];  // (cos, -sin) of 2 pi p q / R
            A.x += sp[q - 1].x * w.x;
            A.y += sp[q - 1].y * w.x;
            B.x -= sm[q - 1].x * w.y;
            B.y -= sm[q - 1].y * w.y;
        }
        const Cx<T> iB = sign < 0 ? Cx<T>{B.y, -B.x} : Cx<T>{-B.y, B.x};  // sign i B
        out[o + p * Ns] = cadd(A, iB);
        out[o + (R - p) * Ns] = csub(A, iB);
    }
}

// The same for any odd prime R up to 64 (kept out of line: loops not unrolled).
template <typename T>
__device__ __noinline__ void odd_radix_any(const Cx<T> *in, Cx<T> *out, int j, int m, int kt, int o, int Ns, int R,
                                           const Cx<T> *tw, int sign) {
    const int h = (R - 1) / 2;
    const Cx<T> v0 = in[j];
    Cx<T> y0 = v0;
    for (int q = 1; q <= h; q++) y0 = cadd(y0, cadd(cmul(in[j + q * m], twid<T>(tw, q * kt, sign)),
                                                    cmul(in[j + (R - q) * m], twid<T>(tw, (R - q) * kt, sign))));
    out[o] = y0;
    for (int p = 1; p <= h; p++) {
        Cx<T> A = v0, B = {T(0), T(0)};
        int e = 0;  // p q mod R
        for (int q = 1; q <= h; q++) {
            e += p;
            if (e >= R) e -= R;
            const Cx<T> u = cmul(in[j + q * m], twid<T>(tw, q * kt, sign));
            const Cx<T> v = cmul(in[j + (R - q) * m], twid<T>(tw, (R - q) * kt, sign));
            const Cx<T> w = tw[e * m];
            A.x += (u.x + v.x) * w.x;
            A.y += (u.y + v.y) * w.x;
            B.x -= (u.x - v.x) * w.y;
            B.y -= (u.y - v.y) * w.y;
        }
        const Cx<T> iB = sign < 0 ? Cx<T>{B.y, -B.x} : Cx<T>{-B.y, B.x};
        out[o + p * Ns] = cadd(A, iB);
        out[o + (R - p) * Ns] = csub(A, iB);
    }
}

// Stockham stages over `lines` lines of length ax.n in shared memory: line l
// at a + l * ls, scratch b alike.  Returns the buffer holding the result.
// Every thread of the block takes part (barriers between stages).  Stage
// twiddle exponents r k n / (Ns R) stay below n (r < R, k < Ns).  An odd
// radix R is a direct DFT with the terms q and R - q paired:
//   y_p     = v_0 + sum_q (v_q + v_{R-q}) cos(2 pi p q / R) + sign i (v_q - v_{R-q}) sin(2 pi p q / R)
//   y_{R-p} = the same with the sine terms negated (q, p = 1 .. (R-1)/2),
// a quarter of the multiplications of the plain DFT.
template <typename T>
__device__ Cx<T> *fft_smem(Cx<T> *a, Cx<T> *b, int ls, int lines, const FftAxis &ax, const Cx<T> *tw, int sign) {
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
                    if (r) v[r] = cmul(v[r], twid<T>(tw, r * k * tscale, sign));
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
                const Cx<T> v0 = in[j], v1 = cmul(in[j + m], twid<T>(tw, k * tscale, sign));
                out[o] = cadd(v0, v1);
                out[o + Ns] = csub(v0, v1);
            } else if (R == 3) {
                odd_radix<T, 3>(in, out, j, m, k * tscale, o, Ns, tw, sign);
            } else if (R == 5) {
                odd_radix<T, 5>(in, out, j, m, k * tscale, o, Ns, tw, sign);
            } else if (R == 7) {
                odd_radix<T, 7>(in, out, j, m, k * tscale, o, Ns, tw, sign);
            } else {  // another odd prime up to 64
                odd_radix_any<T>(in, out, j, m, k * tscale, o, Ns, R, tw, sign);
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

// tw[t] = exp(-2 pi i t / n), t < n, in FP64 and rounded to FP32
__global__ void k_twiddles(Cx<double> *tw, Cx<float> *tw32, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)n, &s, &c);
        tw[t] = Cx<double>{c, s};
        tw32[t] = Cx<float>{(float)c, (float)s};
    }
}

// x forward: rows 2p and 2p + 1 of the real field (rows of length nx, row
// (z, y) = z ny + y), packed as one complex row, transformed and separated
// into their half spectra A_k = (Z_k + conj Z_{-k}) / 2,
// B_k = (Z_k - conj Z_{-k}) / 2i, k = 0 .. nx/2.  An odd row count pairs the
// last row with zeros.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_fwd(const T *__restrict__ R, Cx<T> *__restrict__ S, FftAxis ax,
                                                   const Cx<T> *__restrict__ tw, int64_t n_rows, int ppb) {
    extern __shared__ __align__(16) unsigned char smem_fft[];
    const int nx = ax.n, nxh = nx / 2 + 1;
    const int64_t n_pairs = (n_rows + 1) / 2;
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_fft), *b = a + ppb * nx;
    for (int64_t p0 = (int64_t)blockIdx.x * ppb; p0 < n_pairs; p0 += (int64_t)gridDim.x * ppb) {
        const int np = (int)min((int64_t)ppb, n_pairs - p0);
        for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
            const int l = i / nx, x = i - l * nx;
            const int64_t row = 2 * (p0 + l);
            a[l * nx + x] = Cx<T>{R[row * nx + x], row + 1 < n_rows ? R[(row + 1) * nx + x] : T(0)};
        }
        __syncthreads();
        const Cx<T> *r = fft_smem(a, b, nx, np, ax, tw, -1);
        for (int i = threadIdx.x; i < np * nxh; i += blockDim.x) {
            const int l = i / nxh, k = i - l * nxh;
            const Cx<T> z = r[l * nx + k], w = r[l * nx + (k ? nx - k : 0)];
            const int64_t row = 2 * (p0 + l);
            S[row * nxh + k] = Cx<T>{(z.x + w.x) * T(0.5), (z.y - w.y) * T(0.5)};
            if (row + 1 < n_rows) S[(row + 1) * nxh + k] = Cx<T>{(z.y + w.y) * T(0.5), (w.x - z.x) * T(0.5)};
        }
        __syncthreads();
    }
}

// x inverse: the half spectra of rows 2p and 2p + 1 combined as Z = A + iB
// (full length by Hermitian symmetry), one inverse transform; its real and
// imaginary parts are the two rows (unnormalised; an odd row count takes
// B = 0 for the missing last row).
template <typename T>
__global__ void __launch_bounds__(256) k_fft_x_inv(const Cx<T> *__restrict__ S, T *__restrict__ R, FftAxis ax,
                                                   const Cx<T> *__restrict__ tw, int64_t n_rows, int ppb) {
    extern __shared__ __align__(16) unsigned char smem_fft[];
    const int nx = ax.n, nxh = nx / 2 + 1;
    const int64_t n_pairs = (n_rows + 1) / 2;
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_fft), *b = a + ppb * nx;
    for (int64_t p0 = (int64_t)blockIdx.x * ppb; p0 < n_pairs; p0 += (int64_t)gridDim.x * ppb) {
        const int np = (int)min((int64_t)ppb, n_pairs - p0);
        for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
            const int l = i / nx, k = i - l * nx;
            const int64_t row = 2 * (p0 + l);
            const bool two = row + 1 < n_rows;
            Cx<T> A, B = {T(0), T(0)};
            if (k < nxh) {
                A = S[row * nxh + k];
                if (two) B = S[(row + 1) * nxh + k];
            } else {  // conjugates of the mirrored columns
                A = S[row * nxh + (nx - k)];
                if (two) B = S[(row + 1) * nxh + (nx - k)];
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
            if (row + 1 < n_rows) R[(row + 1) * nx + x] = r[l * nx + x].y;
        }
        __syncthreads();
    }
}

// Column transforms of the spectrum S [nz][ny][nxh] along y (axis 1) or z
// (axis 2), in tiles of tw_w consecutive k_x of one line position (z for y
// columns, y for z columns), coalesced along k_x.  green (z only): forward,
// then 1: times scale / lambda_k (the (0,0,0) mode zeroed), or 2: times the
// spectrum gk [nz][ny][nxh] and scale (the product in FP64), then inverse.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_col(Cx<T> *__restrict__ S, FftAxis ax, const Cx<T> *__restrict__ tw,
                                                 int axis, int nxh, int ny, int nz, int tw_w, int sign, int green,
                                                 const double *__restrict__ lam1, double scale,
                                                 const Cx<T> *__restrict__ gk) {
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
                if (green == 2) {
                    const Cx<T> b = gk[((int64_t)e * ny + o) * nxh + kx];
                    const double re = (double)v.x * b.x - (double)v.y * b.y, im = (double)v.x * b.y + (double)v.y * b.x;
                    v.x = (T)(re * scale);
                    v.y = (T)(im * scale);
                } else if (kx == 0 && o == 0 && e == 0) {
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

// Twiddle tables of the three axes (made once per size) and the kernels'
// shared-memory opt-in.
static amr_status fft_setup(amr_hydro_ctx *c, int nx, int ny, int nz, cudaStream_t s) {
    amr_status st;
    if (c->fft_tw_n[0] != nx || c->fft_tw_n[1] != ny || c->fft_tw_n[2] != nz) {
        // FP64 tables of the three axes, then their FP32 copies
        const int nt = nx + ny + nz;
        if ((st = c->fft_tw.reserve(3 * (size_t)nt))) return st;
        Cx<double> *t = reinterpret_cast<Cx<double> *>(c->fft_tw.p);
        Cx<float> *t32 = reinterpret_cast<Cx<float> *>(t + nt);
        k_twiddles<<<(nx + 255) / 256, 256, 0, s>>>(t, t32, nx);
        k_twiddles<<<(ny + 255) / 256, 256, 0, s>>>(t + nx, t32 + nx, ny);
        k_twiddles<<<(nz + 255) / 256, 256, 0, s>>>(t + nx + ny, t32 + nx + ny, nz);
        if ((st = cuda_fail(cudaGetLastError(), "k_twiddles"))) return st;
        c->fft_tw_n[0] = nx;
        c->fft_tw_n[1] = ny;
        c->fft_tw_n[2] = nz;
    }
    static DeviceOnce once;
    return once_per_device(once, [] {
        amr_status e;
        if ((e = set_smem((const void *)k_fft_x_fwd<double>)) || (e = set_smem((const void *)k_fft_x_inv<double>)) ||
            (e = set_smem((const void *)k_fft_col<double>)) || (e = set_smem((const void *)k_fft_x_fwd<float>)) ||
            (e = set_smem((const void *)k_fft_x_inv<float>)) || (e = set_smem((const void *)k_fft_col<float>)))
            return e;
        return AMR_OK;
    });
}

// The passes over a [nz][ny][nx] real field R and its half spectrum S
// [nz][ny][nx/2+1]; plane ranges [z0, z0 + planes) for the x and y passes.
template <typename T>
struct FftPasses {
    amr_hydro_ctx *c;
    FftAxis ax, ay, az;
    const Cx<T> *twx, *twy, *twz;
    int nx, ny, nz, nxh, ppb, wy, wz, grid;
    cudaStream_t s;
    bool init(amr_hydro_ctx *c_, int nx_, int ny_, int nz_, cudaStream_t s_) {
        c = c_;
        nx = nx_;
        ny = ny_;
        nz = nz_;
        s = s_;
        if (nx % 2 || !fft_factor(nx, ax) || !fft_factor(ny, ay) || !fft_factor(nz, az)) return false;
        const Cx<double> *t64 = reinterpret_cast<const Cx<double> *>(c->fft_tw.p);
        if constexpr (sizeof(T) == sizeof(double)) twx = t64;
        else twx = reinterpret_cast<const Cx<float> *>(t64 + nx + ny + nz);
        twy = twx + nx;
        twz = twy + ny;
        nxh = nx / 2 + 1;
        // lines per CTA: about 2048 points of work for 256 threads; column
        // tiles of at least 64-byte row segments (coalescing); two buffers of
        // at most 160 KB of shared memory
        constexpr size_t SMAX = 160 * 1024;
        ppb = 2048 / nx;
        ppb = ppb < 1 ? 1 : (ppb > 16 ? 16 : ppb);
        while (ppb > 1 && 2 * (size_t)ppb * nx * sizeof(Cx<T>) > SMAX) ppb--;
        auto col_w = [SMAX](int n) {
            const int wmin = sizeof(T) == sizeof(double) ? 4 : 8;
            int w = 2048 / n;
            w = w < wmin ? wmin : (w > 16 ? 16 : w);
            while (w > 1 && 2 * (size_t)w * n * sizeof(Cx<T>) > SMAX) w--;
            return w;
        };
        wy = col_w(ny);
        wz = col_w(nz);
        grid = c->n_sm * 4;
        return true;
    }
    amr_status x(T *R, Cx<T> *S, int z0, int planes, bool forward) const {
        const size_t sx = 2 * (size_t)ppb * nx * sizeof(Cx<T>);
        const int64_t rows = (int64_t)planes * ny;
        if (forward) k_fft_x_fwd<T><<<grid, 256, sx, s>>>(R + (int64_t)z0 * ny * nx, S + (int64_t)z0 * ny * nxh, ax,
                                                         twx, rows, ppb);
        else k_fft_x_inv<T><<<grid, 256, sx, s>>>(S + (int64_t)z0 * ny * nxh, R + (int64_t)z0 * ny * nx, ax, twx, rows,
                                                  ppb);
        return cuda_fail(cudaGetLastError(), "fft x pass");
    }
    amr_status y(Cx<T> *S, int z0, int planes, int sign) const {
        k_fft_col<T><<<grid, 256, 2 * (size_t)wy * ny * sizeof(Cx<T>), s>>>(S + (int64_t)z0 * ny * nxh, ay, twy, 1, nxh,
                                                                            ny, planes, wy, sign, 0, nullptr, 0.0,
                                                                            nullptr);
        return cuda_fail(cudaGetLastError(), "fft y pass");
    }
    amr_status z(Cx<T> *S, int sign, int green, const double *lam1, double scale, const Cx<T> *gk) const {
        k_fft_col<T><<<grid, 256, 2 * (size_t)wz * nz * sizeof(Cx<T>), s>>>(S, az, twz, 2, nxh, ny, nz, wz, sign,
                                                                            green, lam1, scale, gk);
        return cuda_fail(cudaGetLastError(), "fft z pass");
    }
};

template <typename T>
amr_status fft_poisson_periodic(amr_hydro_ctx *c, T *R, int nx, int ny, int nz, const double *lam1, double scale,
                                void *spec, cudaStream_t s) {
    amr_status st;
    if ((st = fft_setup(c, nx, ny, nz, s))) return st;
    FftPasses<T> F;
    if (!F.init(c, nx, ny, nz, s)) return AMR_E_INVAL;
    Cx<T> *S = reinterpret_cast<Cx<T> *>(spec);
    if ((st = F.x(R, S, 0, nz, true)) || (st = F.y(S, 0, nz, -1)) || (st = F.z(S, -1, 1, lam1, scale, nullptr)) ||
        (st = F.y(S, 0, nz, +1)) || (st = F.x(R, S, 0, nz, false)))
        return st;
    return AMR_OK;
}

template <typename T>
amr_status fft_forward_full(amr_hydro_ctx *c, T *R, int mx, int my, int mz, void *spec, cudaStream_t s) {
    amr_status st;
    if ((st = fft_setup(c, mx, my, mz, s))) return st;
    FftPasses<T> F;
    if (!F.init(c, mx, my, mz, s)) return AMR_E_INVAL;
    Cx<T> *S = reinterpret_cast<Cx<T> *>(spec);
    if ((st = F.x(R, S, 0, mz, true)) || (st = F.y(S, 0, mz, -1)) || (st = F.z(S, -1, 0, nullptr, 0.0, nullptr)))
        return st;
    return AMR_OK;
}

template <typename T>
amr_status fft_convolve_isolated(amr_hydro_ctx *c, T *R, int mx, int my, int mz, int nz, const void *gk,
                                 double scale, void *spec, cudaStream_t s) {
    amr_status st;
    if (nz + 2 > mz - 2) return AMR_E_INVAL;
    if ((st = fft_setup(c, mx, my, mz, s))) return st;
    FftPasses<T> F;
    if (!F.init(c, mx, my, mz, s)) return AMR_E_INVAL;
    Cx<T> *S = reinterpret_cast<Cx<T> *>(spec);
    const int64_t plane_c = (int64_t)my * F.nxh;
    // planes z >= nz of the field are zero: so are those of its (y, x) spectrum
    if ((st = cuda_fail(cudaMemsetAsync(S + nz * plane_c, 0, sizeof(Cx<T>) * (mz - nz) * plane_c, s),
                        "memset spectrum")))
        return st;
    if ((st = F.x(R, S, 0, nz, true)) || (st = F.y(S, 0, nz, -1)) ||
        (st = F.z(S, -1, 2, nullptr, scale, reinterpret_cast<const Cx<T> *>(gk))) ||
        (st = F.y(S, 0, nz + 2, +1)) || (st = F.y(S, mz - 2, 2, +1)) || (st = F.x(R, S, 0, nz + 2, false)) ||
        (st = F.x(R, S, mz - 2, 2, false)))
        return st;
    return AMR_OK;
}

template amr_status fft_poisson_periodic<double>(amr_hydro_ctx *, double *, int, int, int, const double *, double,
                                                 void *, cudaStream_t);
template amr_status fft_poisson_periodic<float>(amr_hydro_ctx *, float *, int, int, int, const double *, double,
                                                void *, cudaStream_t);
template amr_status fft_forward_full<double>(amr_hydro_ctx *, double *, int, int, int, void *, cudaStream_t);
template amr_status fft_forward_full<float>(amr_hydro_ctx *, float *, int, int, int, void *, cudaStream_t);
template amr_status fft_convolve_isolated<double>(amr_hydro_ctx *, double *, int, int, int, int, const void *, double,
                                                  void *, cudaStream_t);
template amr_status fft_convolve_isolated<float>(amr_hydro_ctx *, float *, int, int, int, int, const void *, double,
                                                 void *, cudaStream_t);

}  // namespace amrh
