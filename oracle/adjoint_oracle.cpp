// adjoint_oracle.cpp -- discrete adjoint and tangent of one oracle step
// (test infrastructure, like the rest of oracle/; the paper has no adjoint).
//
// hydro_oracle.c is compiled unchanged as C++ twice:
//   * namespace rev: with `double` a reverse-mode number that records every
//     operation and its partial derivatives on a tape; sweeping the tape
//     backwards gives lam_n = (dU^{n+1}/dU^n)^T lam_{n+1};
//   * namespace fwd: with `double` a dual number (value, tangent); one pass
//     gives J v.
// dt, dh and gamma enter as constants (dt frozen).  Branches (limiter sign
// tests, min/max of the wave speeds, the HLLC region) are those the forward
// evaluation takes, so at a kink the derivative of the taken branch is used.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <vector>

namespace rev {
struct Node {
    int a, b;
    double da, db;
};
static std::vector<Node> *tape = nullptr;
struct AD {
    double v;
    int id;  // tape node, -1 for a constant
    AD() = default;
    AD(double x) : v(x), id(-1) {}
};
inline AD node(double v, const AD &a, double da, const AD &b, double db) {
    AD r;
    r.v = v;
    if (a.id < 0 && b.id < 0) {
        r.id = -1;
        return r;
    }
    tape->push_back(Node{a.id, b.id, da, db});
    r.id = (int)tape->size() - 1;
    return r;
}
inline AD leaf(double v) {
    tape->push_back(Node{-1, -1, 0.0, 0.0});
    AD r;
    r.v = v;
    r.id = (int)tape->size() - 1;
    return r;
}
static const AD none(0.0);
inline AD operator+(const AD &a, const AD &b) { return node(a.v + b.v, a, 1.0, b, 1.0); }
inline AD operator-(const AD &a, const AD &b) { return node(a.v - b.v, a, 1.0, b, -1.0); }
inline AD operator*(const AD &a, const AD &b) { return node(a.v * b.v, a, b.v, b, a.v); }
inline AD operator/(const AD &a, const AD &b) { return node(a.v / b.v, a, 1.0 / b.v, b, -a.v / (b.v * b.v)); }
inline AD operator-(const AD &a) { return node(-a.v, a, -1.0, none, 0.0); }
inline AD &operator+=(AD &a, const AD &b) { return a = a + b; }
inline AD &operator-=(AD &a, const AD &b) { return a = a - b; }
inline AD &operator*=(AD &a, const AD &b) { return a = a * b; }
inline bool operator<(const AD &a, const AD &b) { return a.v < b.v; }
inline bool operator>(const AD &a, const AD &b) { return a.v > b.v; }
inline bool operator<=(const AD &a, const AD &b) { return a.v <= b.v; }
inline bool operator>=(const AD &a, const AD &b) { return a.v >= b.v; }
inline AD sqrt(const AD &a) {
    const double s = std::sqrt(a.v);
    return node(s, a, 0.5 / s, none, 0.0);
}
inline AD fabs(const AD &a) { return node(std::fabs(a.v), a, a.v < 0 ? -1.0 : 1.0, none, 0.0); }
inline AD pow(const AD &a, const AD &b) {
    const double p = std::pow(a.v, b.v);
    return node(p, a, b.v * std::pow(a.v, b.v - 1.0), b, p * std::log(a.v));
}
#define double AD
#include "hydro_oracle.c"
#undef double
}  // namespace rev

namespace fwd {
struct Dual {
    double v, d;
    Dual() = default;
    Dual(double x) : v(x), d(0.0) {}
    Dual(double x, double t) : v(x), d(t) {}
};
inline Dual operator+(const Dual &a, const Dual &b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual &a, const Dual &b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(const Dual &a, const Dual &b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual &a, const Dual &b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
inline Dual &operator+=(Dual &a, const Dual &b) { return a = a + b; }
inline Dual &operator-=(Dual &a, const Dual &b) { return a = a - b; }
inline Dual &operator*=(Dual &a, const Dual &b) { return a = a * b; }
inline bool operator<(const Dual &a, const Dual &b) { return a.v < b.v; }
inline bool operator>(const Dual &a, const Dual &b) { return a.v > b.v; }
inline bool operator<=(const Dual &a, const Dual &b) { return a.v <= b.v; }
inline bool operator>=(const Dual &a, const Dual &b) { return a.v >= b.v; }
inline Dual sqrt(const Dual &a) {
    const double s = std::sqrt(a.v);
    return Dual(s, a.d * 0.5 / s);
}
inline Dual fabs(const Dual &a) { return a.v < 0 ? Dual(-a.v, -a.d) : a; }
inline Dual pow(const Dual &a, const Dual &b) {
    const double p = std::pow(a.v, b.v);
    return Dual(p, a.d * b.v * std::pow(a.v, b.v - 1.0) + b.d * p * std::log(a.v));
}
#define double Dual
#include "hydro_oracle.c"
#undef double
}  // namespace fwd

// lam_n = (dS/dU)^T lam_np1 for one periodic step S of size dt (arrays
// [5][nz][ny][nx]).
extern "C" void or_adj_step(const double *U, const double *lam_np1, double *lam_n, int nx, int ny, int nz,
                            double dh, double dt, double gamma) {
    const int64_t n = 5LL * nx * ny * nz;
    std::vector<rev::Node> t;
    t.reserve((size_t)n * 260);
    rev::tape = &t;
    std::vector<rev::AD> u(n), un(n);
    for (int64_t i = 0; i < n; i++) u[i] = rev::leaf(U[i]);
    rev::or_step_periodic_fx(u.data(), un.data(), nx, ny, nz, rev::AD(dh), rev::AD(dt), rev::AD(gamma), nullptr);
    std::vector<double> adj(t.size(), 0.0);
    for (int64_t i = 0; i < n; i++)
        if (un[i].id >= 0) adj[un[i].id] += lam_np1[i];
    for (int64_t k = (int64_t)t.size() - 1; k >= 0; k--) {
        const double g = adj[k];
        if (g == 0.0) continue;
        const rev::Node &nd = t[k];
        if (nd.a >= 0) adj[nd.a] += nd.da * g;
        if (nd.b >= 0) adj[nd.b] += nd.db * g;
    }
    for (int64_t i = 0; i < n; i++) lam_n[i] = adj[u[i].id];
    rev::tape = nullptr;
}

// Jv = (dS/dU) v for one periodic step.
extern "C" void or_jvp_step(const double *U, const double *V, double *JV, int nx, int ny, int nz, double dh,
                            double dt, double gamma) {
    const int64_t n = 5LL * nx * ny * nz;
    std::vector<fwd::Dual> u(n), un(n);
    for (int64_t i = 0; i < n; i++) u[i] = fwd::Dual(U[i], V[i]);
    fwd::or_step_periodic_fx(u.data(), un.data(), nx, ny, nz, fwd::Dual(dh), fwd::Dual(dt), fwd::Dual(gamma),
                             nullptr);
    for (int64_t i = 0; i < n; i++) JV[i] = un[i].d;
}

// Transposed Jacobian of one HLLC flux evaluation: lamUL, lamUR =
// (dF/dUL)^T lamF, (dF/dUR)^T lamF, for a face normal to d.
extern "C" void or_adj_hllc(const double *UL, const double *UR, int d, double gamma, const double *lamF,
                            double *lamUL, double *lamUR) {
    std::vector<rev::Node> t;
    rev::tape = &t;
    rev::AD uL[5], uR[5], F[5];
    for (int v = 0; v < 5; v++) uL[v] = rev::leaf(UL[v]);
    for (int v = 0; v < 5; v++) uR[v] = rev::leaf(UR[v]);
    rev::or_hllc(uL, uR, d, rev::AD(gamma), F);
    std::vector<double> adj(t.size(), 0.0);
    for (int v = 0; v < 5; v++)
        if (F[v].id >= 0) adj[F[v].id] += lamF[v];
    for (int64_t k = (int64_t)t.size() - 1; k >= 0; k--) {
        const double g = adj[k];
        if (g == 0.0) continue;
        if (t[k].a >= 0) adj[t[k].a] += t[k].da * g;
        if (t[k].b >= 0) adj[t[k].b] += t[k].db * g;
    }
    for (int v = 0; v < 5; v++) {
        lamUL[v] = adj[uL[v].id];
        lamUR[v] = adj[uR[v].id];
    }
    rev::tape = nullptr;
}
