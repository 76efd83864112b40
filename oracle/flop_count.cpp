// flop_count.cpp -- instrumented count of the oracle's floating-point
// operations per cell update (test infrastructure, like the rest of oracle/).
//
// hydro_oracle.c is compiled unchanged as C++ with `double` replaced by a
// counting number type, then one periodic step plus one Eq. (CFL2) speed
// reduction is run on a small grid.  The dense oracle evaluates every piece
// of the scheme exactly once per cell (one primitive conversion, one Hancock
// cell, three HLLC faces, one update, one signal speed), so the counts per
// cell are the method's algorithmic operation counts with no ghost-zone
// redundancy.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

namespace fc {
struct Ops {
    long long add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0, other = 0;
};
static Ops ops;
struct Counted {
    double v;
    Counted() = default;
    Counted(double x) : v(x) {}
    Counted &operator+=(Counted b) { ops.add++; v += b.v; return *this; }
    Counted &operator-=(Counted b) { ops.add++; v -= b.v; return *this; }
    Counted &operator*=(Counted b) { ops.mul++; v *= b.v; return *this; }
    Counted operator-() const { return Counted(-v); }  // sign flip: not an arithmetic op
};
inline Counted operator+(Counted a, Counted b) { ops.add++; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ops.add++; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { ops.mul++; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ops.div++; return Counted(a.v / b.v); }
inline bool operator<(Counted a, Counted b) { ops.cmp++; return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { ops.cmp++; return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { ops.cmp++; return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { ops.cmp++; return a.v >= b.v; }
inline Counted sqrt(Counted a) { ops.sqrt++; return Counted(std::sqrt(a.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }  // sign clear: free
inline Counted pow(Counted a, Counted b) { ops.other++; return Counted(std::pow(a.v, b.v)); }
}  // namespace fc
using fc::Counted;
using fc::sqrt;
using fc::fabs;
using fc::pow;

#define double Counted
#include "hydro_oracle.c"
#undef double

// out[0..5] = add/sub, mul, div, sqrt, compare, other operations of one step
// per cell; out[6..11] the same for the Eq. (CFL2) signal-speed reduction.
extern "C" void or_count_flops(const double *U_in, int nx, int ny, int nz, double gamma, double *out) {
    const int64_t n = (int64_t)nx * ny * nz;
    Counted *U = (Counted *)std::malloc(sizeof(Counted) * 5 * n);
    Counted *Un = (Counted *)std::malloc(sizeof(Counted) * 5 * n);
    for (int64_t i = 0; i < 5 * n; i++) U[i] = Counted(U_in[i]);
    Counted s = or_max_speed(U, n, Counted(gamma));
    Counted dt = Counted(0.25 / nx) / s;  // not counted below: reset first
    fc::ops = fc::Ops();
    or_step_periodic(U, Un, nx, ny, nz, Counted(1.0 / nx), dt, Counted(gamma));
    fc::Ops a = fc::ops;
    fc::ops = fc::Ops();
    or_max_speed(Un, n, Counted(gamma));
    fc::Ops b = fc::ops;
    const long long *pa = &a.add, *pb = &b.add;
    for (int k = 0; k < 6; k++) {
        out[k] = (double)pa[k] / n;
        out[6 + k] = (double)pb[k] / n;
    }
    std::free(U);
    std::free(Un);
}
