// hydro_math.cuh -- pointwise device arithmetic of the MUSCL-Hancock / HLLC
// update (GAMER-2 section 2.2), templated on the compute type `real`
// (double for AMR_FP64, float for AMR_FP32_ACC64).
//
// Conserved U = (rho, rho vx, rho vy, rho vz, E); primitive
// W = (rho, vx, vy, vz, P); ideal gas P = (gamma-1)(E - rho|v|^2/2).
#pragma once
#include <cstdint>

namespace amrh {

constexpr int NV = 5;

// ---- reciprocal, reciprocal square root, square root -------------------------
//
// FP64: on this GPU the FP64 pipe issues 2 operations per clock per SM, and an
// IEEE division costs about nine of them.  The reciprocal is instead seeded by
// the special-function unit's approximate reciprocal (rcp.approx.ftz.f64,
// which runs on a separate, much wider unit, relative error below 2^-20) and
// refined by one third-order step of Householder's method for f(r) = 1/r - x:
// with e = 1 - x r, r <- r (1 + e + e^2) leaves a relative error of e^3
// (below 2^-60, so the result is at the FP64 rounding level) in 3 fused
// multiply-adds, one fewer than two Newton-Raphson steps.  The reciprocal
// square root takes the same route for f(y) = 1/y^2 - x: with e = 1 - x y^2,
// y <- y (1 + e/2 + 3e^2/8) (the binomial series of (1 - e)^(-1/2) to second
// order; error 5e^3/16), 5 operations.  The square root of a positive normal
// x is x * rsqrt_(x) (a few ulp); zeros, subnormals, negative and non-finite
// inputs take CUDA's sqrt.  All three are checked against IEEE division and
// square root in the tests.
// FP32: the hardware approximations (about 1 ulp), inside the FP32 mode's
// 1e-5 tolerance.
__device__ __forceinline__ double rcp_(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double rsqrt_(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y * y, 1.0);
    return fma(y * e, fma(e, 0.375, 0.5), y);
}
__device__ __forceinline__ double sqrt_(double x) {
    // positive normal: high word in [0x00100000, 0x7fefffff]
    const unsigned hi = (unsigned)__double2hiint(x);
    if (hi - 0x00100000u < 0x7fe00000u) return x * rsqrt_(x);
    return sqrt(x);
}
__device__ __forceinline__ float rcp_(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- FP64 <-> FP32 without the FP64 pipe ---------------------------------------
//
// cvt between double and float issues on the FP64 pipe; in the FP32 mode that
// made conversions the bottleneck, so they are done on the integer units from
// the IEEE-754 bit layouts (sign | exponent | fraction; biases 1023 and 127).
// double -> float: round half away from zero on the first dropped fraction
// bit; magnitudes below 2^-126 flush to zero (the FP32 mode runs with
// flush-to-zero); finite inputs above the float range are not expected.
__device__ __forceinline__ float d2f_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned e = (hi >> 20) & 0x7ffu;
    unsigned r = ((hi << 3) | (lo >> 29)) - (896u << 23);
    r += (lo >> 28) & 1u;
    r = e > 896u ? r : 0u;
    return __uint_as_float(r | (hi & 0x80000000u));
}
// float -> double: exact (flushed float zeros map to signed zeros).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned s = b & 0x80000000u, mag = b & 0x7fffffffu;
    const unsigned hi = mag >= 0x00800000u ? (s | ((mag >> 3) + (896u << 20))) : s;
    const unsigned lo = mag >= 0x00800000u ? (b << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

template <typename real>
__device__ __forceinline__ real to_real(double x);
template <>
__device__ __forceinline__ double to_real<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_real<float>(double x) { return d2f_bits(x); }

// ---- sign tests and ordering on the integer units ----------------------------------
//
// Every FP64 comparison takes a full issue of the narrow FP64 pipe, which sets
// the pace of the FP64 step, so in FP64 the limiter's and the Riemann solver's
// sign tests and min/max read the IEEE-754 bit pattern on the integer units
// instead.  For a non-NaN double with bits b (a signed 64-bit integer):
// x > 0 <=> b > 0 (+0 is 0, -0 is negative); x <= 0 <=> b <= 0;
// x >= 0 <=> b >= 0 or x is -0.  okey(x) flips the magnitude bits of negative
// values, so it orders like x, except that -0 sorts just below +0 (a min/max
// of two zeros of opposite sign may return the other zero).  FP32 keeps the
// ordinary comparisons, which run on the integer/ALU pipe anyway.
__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool le0(double x) { return __double_as_longlong(x) <= 0; }
__device__ __forceinline__ bool ge0(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 || b == (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ double min_(double a, double b) { return okey(a) <= okey(b) ? a : b; }
__device__ __forceinline__ double max_(double a, double b) { return okey(a) >= okey(b) ? a : b; }
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
__device__ __forceinline__ bool le0(float x) { return x <= 0.0f; }
__device__ __forceinline__ bool ge0(float x) { return x >= 0.0f; }
__device__ __forceinline__ float min_(float a, float b) { return (a <= b) ? a : b; }
__device__ __forceinline__ float max_(float a, float b) { return (a >= b) ? a : b; }

// Scheme options (amr_limiter / amr_riemann of the C ABI).
constexpr int LIM_VANLEER = 0, LIM_GMINMOD = 1, LIM_ALBADA = 2, LIM_VL_GMINMOD = 3;
constexpr int RS_HLLC = 0, RS_HLLE = 1, RS_ROE = 2, RS_EXACT = 3;

template <typename real>
struct Gas {
    real gamma, gm1, inv_gm1;
    int lim = LIM_VANLEER, rs = RS_HLLC;  // uniform over a launch: the branches on them never diverge
    real htheta = real(0.75);             // half the generalized minmod coefficient
    int fb = 0;                           // remedies for unphysical results: no flux for an unphysical
                                          // face state, and Roe falls back to HLLE
};

template <typename real>
__device__ __forceinline__ real qnan();
template <>
__device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <>
__device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }

// x > 0 and finite, on the bit pattern (a NaN or +inf fails)
__device__ __forceinline__ bool pos_finite(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool pos_finite(float x) {
    const int b = __float_as_int(x);
    return b > 0 && b < 0x7f800000;
}

// |x| and sign transfer on the bit pattern (integer units)
__device__ __forceinline__ double fabs_(double x) {
    return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double copysign_(double m, double s) {
    return __longlong_as_double(__double_as_longlong(m) | (__double_as_longlong(s) & (long long)0x8000000000000000ULL));
}
__device__ __forceinline__ float fabs_(float x) { return __int_as_float(__float_as_int(x) & 0x7fffffff); }
__device__ __forceinline__ float copysign_(float m, float s) {
    return __int_as_float(__float_as_int(m) | (__float_as_int(s) & (int)0x80000000u));
}

// U -> W; also returns 1/rho for reuse.
template <typename real>
__device__ __forceinline__ real u2w(const real u[NV], real w[NV], const Gas<real> &g) {
    const real ri = rcp_(u[0]);
    w[0] = u[0];
    w[1] = u[1] * ri;
    w[2] = u[2] * ri;
    w[3] = u[3] * ri;
    w[4] = g.gm1 * (u[4] - real(0.5) * u[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
    return ri;
}

// W -> U
template <typename real>
__device__ __forceinline__ void w2u(const real w[NV], real u[NV], const Gas<real> &g) {
    u[0] = w[0];
    u[1] = w[0] * w[1];
    u[2] = w[0] * w[2];
    u[3] = w[0] * w[3];
    u[4] = w[4] * g.inv_gm1 + real(0.5) * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

// Half of the limited slope of the selected limiter, from the one-sided
// differences a = W_i - W_{i-1}, b = W_{i+1} - W_i (0 unless ab > 0):
// van Leer-type ab/(a+b); generalized minmod sign(a) min(t|a|, |a+b|/2, t|b|)/2;
// van Albada-type ab(a+b)/(2(a^2+b^2)); hybrid the smaller in magnitude of
// the first two.  The selects keep a warp convergent, and the limiter branch
// is uniform over a launch.
template <typename real>
__device__ __forceinline__ real half_slope(real a, real b, const Gas<real> &g) {
    const real ab = a * b;
    real h;
    if (g.lim == LIM_VANLEER) {
        h = ab * rcp_(a + b);
    } else if (g.lim == LIM_ALBADA) {
        h = ab * (a + b) * rcp_(real(2) * (a * a + b * b));
    } else {
        real m = min_(min_(g.htheta * fabs_(a), g.htheta * fabs_(b)), real(0.25) * fabs_(a + b));
        if (g.lim == LIM_VL_GMINMOD) m = min_(m, fabs_(ab * rcp_(a + b)));
        h = copysign_(m, a);
    }
    return gt0(ab) ? h : real(0);
}

// Physical flux along D of a state known in both forms (w, u).
template <int D, typename real>
__device__ __forceinline__ void phys_flux(const real w[NV], const real u[NV], real f[NV]) {
    const real vn = w[1 + D];
    f[0] = u[0] * vn;
    f[1] = u[1] * vn;
    f[2] = u[2] * vn;
    f[3] = u[3] * vn;
    f[1 + D] += w[4];
    f[4] = (u[4] + w[4]) * vn;
}

// ---- exact Riemann solver (Toro 2009 ch. 4) --------------------------------------
//
// Pressure function of one side K for a trial star pressure p: a shock when
// p > p_K, a rarefaction otherwise; f and df/dp.
template <typename real>
__device__ __forceinline__ void pressure_fk(real p, real rk, real pk, real ck, const Gas<real> &g, real &f,
                                            real &df) {
    if (p > pk) {
        const real A = real(2) / ((g.gamma + real(1)) * rk), B = g.gm1 / (g.gamma + real(1)) * pk;
        const real q = sqrt_(A / (p + B));
        f = (p - pk) * q;
        df = q * (real(1) - real(0.5) * (p - pk) / (B + p));
    } else {
        const real e = g.gm1 / (real(2) * g.gamma);
        f = real(2) * ck / g.gm1 * (pow(p / pk, e) - real(1));
        df = pow(p / pk, -(g.gamma + real(1)) / (real(2) * g.gamma)) / (rk * ck);
    }
}

// Godunov flux: the physical flux of the exact solution at x/t = 0.  Star
// pressure by Newton iteration on f_L(p) + f_R(p) + u_R - u_L = 0 from the
// arithmetic-mean pressure (relative change below 1e-15 in FP64, 1e-7 in
// FP32, at most 60 iterations); transverse velocities from the side of the
// contact x/t = 0 lies on (the left one when the contact is at rest).
template <int D, typename real>
__device__ __noinline__ void exact_flux(const real uL[NV], const real uR[NV], real F[NV], const Gas<real> &g) {
    real wL[NV], wR[NV];
    u2w(uL, wL, g);
    u2w(uR, wR, g);
    const real rl = wL[0], ul = wL[1 + D], pl = wL[4];
    const real rr = wR[0], ur = wR[1 + D], pr = wR[4];
    if (g.fb && !(pos_finite(rl) && pos_finite(pl) && pos_finite(rr) && pos_finite(pr))) {
#pragma unroll
        for (int v = 0; v < NV; v++) F[v] = qnan<real>();  // no flux (as face_flux)
        return;
    }
    const real cl = sqrt_(g.gamma * pl / rl), cr = sqrt_(g.gamma * pr / rr);
    const real tol = sizeof(real) == sizeof(double) ? real(1e-15) : real(1e-7);
    real p = real(0.5) * (pl + pr), fl, dfl, fr, dfr;
    for (int it = 0; it < 60; it++) {
        pressure_fk(p, rl, pl, cl, g, fl, dfl);
        pressure_fk(p, rr, pr, cr, g, fr, dfr);
        real pn = p - (fl + fr + (ur - ul)) / (dfl + dfr);
        if (!(pn > real(0))) pn = real(1e-14) * p;
        const real change = real(2) * fabs_(pn - p) / (pn + p);
        p = pn;
        if (change < tol) break;
    }
    pressure_fk(p, rl, pl, cl, g, fl, dfl);
    pressure_fk(p, rr, pr, cr, g, fr, dfr);
    const real ps = p, us = real(0.5) * (ul + ur) + real(0.5) * (fr - fl);
    const real g1 = g.gm1 / (g.gamma + real(1));
    real r, v, q;
    if (us >= real(0)) {  // x/t = 0 left of the contact
        if (ps > pl) {
            const real S = ul - cl * sqrt_((g.gamma + real(1)) / (real(2) * g.gamma) * ps / pl +
                                           g.gm1 / (real(2) * g.gamma));
            if (S >= real(0)) { r = rl; v = ul; q = pl; }
            else { r = rl * (ps / pl + g1) / (g1 * ps / pl + real(1)); v = us; q = ps; }
        } else {
            const real cs = cl * pow(ps / pl, g.gm1 / (real(2) * g.gamma));
            if (ul - cl >= real(0)) { r = rl; v = ul; q = pl; }
            else if (us - cs <= real(0)) { r = rl * pow(ps / pl, real(1) / g.gamma); v = us; q = ps; }
            else {
                const real k = real(2) / (g.gamma + real(1)) + g1 / cl * ul;
                r = rl * pow(k, real(2) / g.gm1);
                v = real(2) / (g.gamma + real(1)) * (cl + real(0.5) * g.gm1 * ul);
                q = pl * pow(k, real(2) * g.gamma / g.gm1);
            }
        }
    } else {  // right of the contact
        if (ps > pr) {
            const real S = ur + cr * sqrt_((g.gamma + real(1)) / (real(2) * g.gamma) * ps / pr +
                                           g.gm1 / (real(2) * g.gamma));
            if (S <= real(0)) { r = rr; v = ur; q = pr; }
            else { r = rr * (ps / pr + g1) / (g1 * ps / pr + real(1)); v = us; q = ps; }
        } else {
            const real cs = cr * pow(ps / pr, g.gm1 / (real(2) * g.gamma));
            if (ur + cr <= real(0)) { r = rr; v = ur; q = pr; }
            else if (us + cs >= real(0)) { r = rr * pow(ps / pr, real(1) / g.gamma); v = us; q = ps; }
            else {
                const real k = real(2) / (g.gamma + real(1)) - g1 / cr * ur;
                r = rr * pow(k, real(2) / g.gm1);
                v = real(2) / (g.gamma + real(1)) * (-cr + real(0.5) * g.gm1 * ur);
                q = pr * pow(k, real(2) * g.gamma / g.gm1);
            }
        }
    }
    const real *wt = us >= real(0) ? wL : wR;
    real w[NV], u[NV];
    w[0] = r;
    w[1] = wt[1];
    w[2] = wt[2];
    w[3] = wt[3];
    w[1 + D] = v;
    w[4] = q;
    w2u(w, u, g);
    phys_flux<D>(w, u, F);
}

// Flux through a face normal to D of the selected Riemann solver:
//   HLLC: Einfeldt/Roe outer speeds, Toro's star states; ties S_L>=0 -> F_L,
//         S_R<=0 -> F_R, S*>=0 -> F*_L;
//   HLLE: the same outer speeds and ties, one intermediate state;
//   Roe:  (F_L + F_R)/2 - (1/2) sum_k |lambda_k| alpha_k K_k with Roe
//         averages, Harten-Hyman entropy fix on the acoustic waves; with
//         g.fb, the HLLE flux when an intermediate state is unphysical;
//   exact: exact_flux above.
// Reciprocals are shared: 1/rho from one reciprocal square root per side,
// which also gives the Roe weight sqrt(rho).
template <int D, typename real>
__device__ __forceinline__ void face_flux(const real uL[NV], const real uR[NV], real F[NV],
                                          const Gas<real> &g) {
    if (g.rs == RS_EXACT) {
        exact_flux<D>(uL, uR, F, g);
        return;
    }
    const real yl = rsqrt_(uL[0]), yr = rsqrt_(uR[0]);  // 1/sqrt(rho)
    const real ril = yl * yl, rir = yr * yr;            // 1/rho
    const real sl = uL[0] * yl, sr = uR[0] * yr;        // sqrt(rho)
    real wL[NV], wR[NV];
    wL[0] = uL[0];
    wL[1] = uL[1] * ril;
    wL[2] = uL[2] * ril;
    wL[3] = uL[3] * ril;
    wL[4] = g.gm1 * (uL[4] - real(0.5) * uL[0] * (wL[1] * wL[1] + wL[2] * wL[2] + wL[3] * wL[3]));
    wR[0] = uR[0];
    wR[1] = uR[1] * rir;
    wR[2] = uR[2] * rir;
    wR[3] = uR[3] * rir;
    wR[4] = g.gm1 * (uR[4] - real(0.5) * uR[0] * (wR[1] * wR[1] + wR[2] * wR[2] + wR[3] * wR[3]));
    const real rl = wL[0], pl = wL[4], ul = wL[1 + D];
    const real rr = wR[0], pr = wR[4], ur = wR[1 + D];
    if (g.fb && !(pos_finite(rl) && pos_finite(pl) && pos_finite(rr) && pos_finite(pr))) {
        // with the remedies on, an unphysical face state has no flux: NaN marks
        // both cells unphysical
#pragma unroll
        for (int v = 0; v < NV; v++) F[v] = qnan<real>();
        return;
    }
    const real cl = sqrt_(g.gamma * pl * ril);
    const real cr = sqrt_(g.gamma * pr * rir);
    const real iw = rcp_(sl + sr);
    const real vtx = (sl * wL[1] + sr * wR[1]) * iw;
    const real vty = (sl * wL[2] + sr * wR[2]) * iw;
    const real vtz = (sl * wL[3] + sr * wR[3]) * iw;
    // Roe-averaged enthalpy (sqrt(rho_L) H_L + sqrt(rho_R) H_R) / (sqrt(rho_L) + sqrt(rho_R))
    // with sqrt(rho) H = (E + P) / sqrt(rho)
    const real ht = ((uL[4] + pl) * yl + (uR[4] + pr) * yr) * iw;
    const real ct = sqrt_(g.gm1 * (ht - real(0.5) * (vtx * vtx + vty * vty + vtz * vtz)));
    const real vtn = D == 0 ? vtx : (D == 1 ? vty : vtz);

    if (g.rs == RS_ROE) {
        real fl[NV], fr[NV];
        phys_flux<D>(wL, uL, fl);
        phys_flux<D>(wR, uR, fr);
        const real vt[3] = {vtx, vty, vtz};
        const real q2 = vtx * vtx + vty * vty + vtz * vtz, a = ct, ra = sl * sr;  // Roe density
        const real ia2 = rcp_(a * a);
        const real dp = pr - pl, dun = ur - ul;
        const real a1 = real(0.5) * (dp - ra * a * dun) * ia2;
        const real a2 = (rr - rl) - dp * ia2;
        const real a5 = real(0.5) * (dp + ra * a * dun) * ia2;
        real l1 = fabs_(vtn - a), l5 = fabs_(vtn + a);
        const real l2 = fabs_(vtn);
        // Harten-Hyman: delta = max(0, lambda~ - lambda(W_L), lambda(W_R) - lambda~)
        real del = max_(max_(real(0), (vtn - a) - (ul - cl)), (ur - cr) - (vtn - a));
        if (l1 < del) l1 = (l1 * l1 + del * del) * rcp_(real(2) * del);
        del = max_(max_(real(0), (vtn + a) - (ul + cl)), (ur + cr) - (vtn + a));
        if (l5 < del) l5 = (l5 * l5 + del * del) * rcp_(real(2) * del);
        const real s15 = l1 * a1 + l2 * a2 + l5 * a5;
        real Dv[NV];
        Dv[0] = s15;
        Dv[1] = s15 * vtx;
        Dv[2] = s15 * vty;
        Dv[3] = s15 * vtz;
        Dv[1 + D] += (l5 * a5 - l1 * a1) * a;
        Dv[4] = l1 * a1 * (ht - vtn * a) + l2 * a2 * real(0.5) * q2 + l5 * a5 * (ht + vtn * a);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (k == D) continue;
            const real sh = l2 * ra * (wR[1 + k] - wL[1 + k]);  // shear wave along k
            Dv[1 + k] += sh;
            Dv[4] += sh * vt[k];
        }
#pragma unroll
        for (int v = 0; v < NV; v++) F[v] = real(0.5) * (fl[v] + fr[v]) - real(0.5) * Dv[v];
        if (!g.fb) return;
        // Remedy (i): the intermediate states U_L + a1 K1 and U_R - a5 K5
        // (K_1,5 = (1, v -/+ a n, H -/+ v_n a)) must have rho > 0 and P > 0,
        // that is 2 rho E > |m|^2; otherwise the face takes the HLLE flux.
        bool ok = pos_finite(a);
#pragma unroll
        for (int s2 = 0; s2 < 2; s2++) {
            const real al = s2 == 0 ? a1 : -a5, sg = s2 == 0 ? real(-1) : real(1);
            const real *u0 = s2 == 0 ? uL : uR;
            real m[3];
#pragma unroll
            for (int k = 0; k < 3; k++) m[k] = u0[1 + k] + al * vt[k];
            m[D] += al * sg * a;
            const real rs2 = u0[0] + al, es = u0[4] + al * (ht + sg * vtn * a);
            ok = ok && pos_finite(rs2) && pos_finite(real(2) * rs2 * es - (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]));
        }
        if (ok) return;
    }

    const real SL = min_(ul - cl, vtn - ct);
    const real SR = max_(ur + cr, vtn + ct);

    if (ge0(SL)) {
        phys_flux<D>(wL, uL, F);
        return;
    }
    if (le0(SR)) {
        phys_flux<D>(wR, uR, F);
        return;
    }
    if (g.rs == RS_HLLE || g.rs == RS_ROE) {  // one intermediate state: (S_R F_L - S_L F_R + S_L S_R (U_R - U_L))/(S_R - S_L)
        real fl[NV], fr[NV];
        phys_flux<D>(wL, uL, fl);
        phys_flux<D>(wR, uR, fr);
        const real ids = rcp_(SR - SL), sls = SL * SR;
#pragma unroll
        for (int v = 0; v < NV; v++) F[v] = (SR * fl[v] - SL * fr[v] + sls * (uR[v] - uL[v])) * ids;
        return;
    }
    const real ml = rl * (SL - ul), mr = rr * (SR - ur);  // mass fluxes relative to the waves
    const real Ss = (pr - pl + ml * ul - mr * ur) * rcp_(ml - mr);
    const bool left = ge0(Ss);
    const real *uK = left ? uL : uR;
    const real *wK = left ? wL : wR;
    const real SK = left ? SL : SR;
    const real mK = left ? ml : mr;
    const real riK = left ? ril : rir;
    const real uKn = wK[1 + D], pK = wK[4];
    real fK[NV];
    phys_flux<D>(wK, uK, fK);
    // Toro's star state U*_K = fac (1, ..., S*, ..., E_K/rho_K + (S* - u_K)(S* + P_K/m_K)),
    // fac = m_K / (S_K - S*); the P_K / m_K term is (S* - u_K) P_K / (S_K - S*)
    // after the factor, so one reciprocal serves both
    const real rsk = rcp_(SK - Ss);
    const real fac = mK * rsk, dS = Ss - uKn;
    real us[NV];
    us[0] = fac;
    us[1] = fac * wK[1];
    us[2] = fac * wK[2];
    us[3] = fac * wK[3];
    us[1 + D] = fac * Ss;
    us[4] = fac * (uK[4] * riK + dS * Ss) + (rsk * dS) * pK;
#pragma unroll
    for (int v = 0; v < NV; v++) F[v] = fK[v] + SK * (us[v] - uK[v]);
}

// Signal speed of Eq. (CFL2), |vx|+|vy|+|vz|+3c_s, or with cfl1 of Eq. (CFL1),
// max(|vx|,|vy|,|vz|)+c_s, of one conserved state, and whether the state is
// physical (rho>0 and P>0, both finite: a NaN from a face state with negative
// pressure counts as unphysical).
template <typename real>
__device__ __forceinline__ real cfl_speed(const real u[NV], const Gas<real> &g, bool &ok, bool cfl1 = false) {
    real w[NV];
    const real ri = u2w(u, w, g);
    ok = pos_finite(w[0]) && pos_finite(w[4]);
    const real cs = sqrt_(g.gamma * w[4] * ri);
    if (cfl1) return max_(max_(fabs(w[1]), fabs(w[2])), fabs(w[3])) + cs;
    return fabs(w[1]) + fabs(w[2]) + fabs(w[3]) + real(3) * cs;
}

}  // namespace amrh
