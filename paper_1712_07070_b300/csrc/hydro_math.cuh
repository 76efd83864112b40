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

// Reciprocal and square root per compute type.  FP64 uses IEEE-rounded
// division and sqrt; FP32 uses the hardware approximations (about 1 ulp),
// well inside the FP32 mode's 1e-5 tolerance.
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float rcp_(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename real>
struct Gas {
    real gamma, gm1, inv_gm1;
};

// U -> W
template <typename real>
__device__ __forceinline__ void u2w(const real u[NV], real w[NV], const Gas<real> &g) {
    const real ri = rcp_(u[0]);
    w[0] = u[0];
    w[1] = u[1] * ri;
    w[2] = u[2] * ri;
    w[3] = u[3] * ri;
    w[4] = g.gm1 * (u[4] - real(0.5) * u[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
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

// Half of the van Leer-type limited slope: vL(a,b)/2 = ab/(a+b) if ab>0.
template <typename real>
__device__ __forceinline__ real half_vanleer(real a, real b) {
    const real ab = a * b;
    return ab > real(0) ? ab * rcp_(a + b) : real(0);
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

// HLLC flux through a face normal to D (Einfeldt/Roe outer speeds, Toro's
// star states; ties: S_L>=0 -> F_L, S_R<=0 -> F_R, S*>=0 -> F*_L).
template <int D, typename real>
__device__ __forceinline__ void hllc(const real uL[NV], const real uR[NV], real F[NV],
                                     const Gas<real> &g) {
    real wL[NV], wR[NV];
    u2w(uL, wL, g);
    u2w(uR, wR, g);
    const real rl = wL[0], pl = wL[4], ul = wL[1 + D];
    const real rr = wR[0], pr = wR[4], ur = wR[1 + D];
    const real cl = sqrt_(g.gamma * pl / rl);
    const real cr = sqrt_(g.gamma * pr / rr);
    const real sl = sqrt_(rl), sr = sqrt_(rr);
    const real iw = rcp_(sl + sr);
    const real vtx = (sl * wL[1] + sr * wR[1]) * iw;
    const real vty = (sl * wL[2] + sr * wR[2]) * iw;
    const real vtz = (sl * wL[3] + sr * wR[3]) * iw;
    const real hl = (uL[4] + pl) / rl, hr = (uR[4] + pr) / rr;
    const real ht = (sl * hl + sr * hr) * iw;
    const real ct = sqrt_(g.gm1 * (ht - real(0.5) * (vtx * vtx + vty * vty + vtz * vtz)));
    const real vtn = D == 0 ? vtx : (D == 1 ? vty : vtz);

    real a = ul - cl, b = vtn - ct;
    const real SL = (a <= b) ? a : b;
    a = ur + cr;
    b = vtn + ct;
    const real SR = (a >= b) ? a : b;

    if (SL >= real(0)) {
        phys_flux<D>(wL, uL, F);
        return;
    }
    if (SR <= real(0)) {
        phys_flux<D>(wR, uR, F);
        return;
    }
    const real Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
                    (rl * (SL - ul) - rr * (SR - ur));
    const bool left = Ss >= real(0);
    const real *uK = left ? uL : uR;
    const real *wK = left ? wL : wR;
    const real SK = left ? SL : SR;
    const real rK = wK[0], uKn = wK[1 + D], pK = wK[4];
    real fK[NV];
    phys_flux<D>(wK, uK, fK);
    const real fac = rK * (SK - uKn) / (SK - Ss);
    real us[NV];
    us[0] = fac;
    us[1] = fac * wK[1];
    us[2] = fac * wK[2];
    us[3] = fac * wK[3];
    us[1 + D] = fac * Ss;
    us[4] = fac * (uK[4] / rK + (Ss - uKn) * (Ss + pK / (rK * (SK - uKn))));
#pragma unroll
    for (int v = 0; v < NV; v++) F[v] = fK[v] + SK * (us[v] - uK[v]);
}

// Signal speed of Eq. (CFL2) of one conserved state, and whether the state is
// physical (rho>0 and P>0).
template <typename real>
__device__ __forceinline__ real cfl_speed(const real u[NV], const Gas<real> &g, bool &ok) {
    real w[NV];
    u2w(u, w, g);
    ok = (w[0] > real(0)) && (w[4] > real(0));
    return fabs(w[1]) + fabs(w[2]) + fabs(w[3]) + real(3) * sqrt_(g.gamma * w[4] * rcp_(w[0]));
}

}  // namespace amrh
