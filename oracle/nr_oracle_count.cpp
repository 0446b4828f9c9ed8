// nr_oracle_count.cpp -- operation-counting build of the oracle.
//
// TEST INFRASTRUCTURE ONLY, like the oracle itself.  It compiles nr_oracle.c
// unchanged as C++ with every `double` replaced by a number type that counts
// the FP64 operations performed on it, so that one right-hand-side evaluation
// (orc_rhs: the BSSN equations of Sec. 2.1 with upwinded advection and
// Kreiss-Oliger dissipation, evaluated in the coordinate basis with generic
// index loops) reports the arithmetic of the method's plain evaluation per
// interior point:
//   add  additions and subtractions (a negation is a sign flip: not counted),
//   mul  multiplications,
//   div  divisions,
//   sqrt square roots,
//   lib  calls of library functions (sin, cos, sinh, cosh, asinh, exp, expm1,
//        log1p, pow, atan2, acos; the oracle evaluates the reference metric at every
//        point from them),
//   cmp  comparisons (not arithmetic; reported for completeness).
// The oracle contains no fused multiply-add and is compiled without contraction,
// so add + mul + div is its FP64 FLOP count with a division counted once.
// Every count is a property of the source: the number type does no arithmetic
// of its own besides the FP64 operation it records.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

namespace {

struct OpCounts {
    long long add, mul, div, sqrt_, lib, cmp;
};
OpCounts g_ops;

// an FP64 value whose operations are counted
struct CD {
    double v;
    constexpr CD() : v(0.0) {}
    constexpr CD(double x) : v(x) {}
    constexpr CD(int x) : v((double)x) {}
    constexpr CD(long x) : v((double)x) {}
    constexpr CD(long long x) : v((double)x) {}
    constexpr CD(unsigned x) : v((double)x) {}
    constexpr CD(unsigned long x) : v((double)x) {}
    constexpr CD(unsigned long long x) : v((double)x) {}
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    explicit operator long long() const { return (long long)v; }
    explicit operator bool() const { return v != 0.0; }
    CD& operator+=(CD b) { ++g_ops.add; v += b.v; return *this; }
    CD& operator-=(CD b) { ++g_ops.add; v -= b.v; return *this; }
    CD& operator*=(CD b) { ++g_ops.mul; v *= b.v; return *this; }
    CD& operator/=(CD b) { ++g_ops.div; v /= b.v; return *this; }
};
static_assert(sizeof(CD) == sizeof(double) && alignof(CD) == alignof(double), "CD must be laid out as a double");

inline CD operator+(CD a, CD b) { ++g_ops.add; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { ++g_ops.add; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { ++g_ops.mul; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { ++g_ops.div; return CD(a.v / b.v); }
inline CD operator-(CD a) { return CD(-a.v); }
inline CD operator+(CD a) { return a; }
inline bool operator<(CD a, CD b) { ++g_ops.cmp; return a.v < b.v; }
inline bool operator>(CD a, CD b) { ++g_ops.cmp; return a.v > b.v; }
inline bool operator<=(CD a, CD b) { ++g_ops.cmp; return a.v <= b.v; }
inline bool operator>=(CD a, CD b) { ++g_ops.cmp; return a.v >= b.v; }
inline bool operator==(CD a, CD b) { ++g_ops.cmp; return a.v == b.v; }
inline bool operator!=(CD a, CD b) { ++g_ops.cmp; return a.v != b.v; }

}  // namespace

// library functions on counted values
inline CD sin(CD x) { ++g_ops.lib; return CD(sin(x.v)); }
inline CD cos(CD x) { ++g_ops.lib; return CD(cos(x.v)); }
inline CD sinh(CD x) { ++g_ops.lib; return CD(sinh(x.v)); }
inline CD cosh(CD x) { ++g_ops.lib; return CD(cosh(x.v)); }
inline CD exp(CD x) { ++g_ops.lib; return CD(exp(x.v)); }
inline CD expm1(CD x) { ++g_ops.lib; return CD(expm1(x.v)); }
inline CD log1p(CD x) { ++g_ops.lib; return CD(log1p(x.v)); }
inline CD acos(CD x) { ++g_ops.lib; return CD(acos(x.v)); }
inline CD asinh(CD x) { ++g_ops.lib; return CD(asinh(x.v)); }
inline CD atan2(CD y, CD x) { ++g_ops.lib; return CD(atan2(y.v, x.v)); }
inline CD pow(CD x, CD y) { ++g_ops.lib; return CD(pow(x.v, y.v)); }
inline CD sqrt(CD x) { ++g_ops.sqrt_; return CD(sqrt(x.v)); }
inline CD fabs(CD x) { return CD(fabs(x.v)); }
inline CD floor(CD x) { return CD(floor(x.v)); }
inline CD round(CD x) { return CD(round(x.v)); }
inline CD nearbyint(CD x) { return CD(nearbyint(x.v)); }
inline CD ldexp(CD x, int e) { ++g_ops.mul; return CD(ldexp(x.v, e)); }

#define double CD
#include "nr_oracle.c"
#undef double

// counts of one orc_rhs over all interior points of the grid described by params (an
// orc_params as the plain oracle takes it; the counting build's copy has the same layout),
// from the 24-gridfunction set gfs into rhs (both 24*T doubles); one thread.
// out: add, mul, div, sqrt, lib, cmp
extern "C" __attribute__((visibility("default"))) int orc_count_rhs(const void* params, const double* gfs,
                                                                   double* rhs, long long out[6])
{
    orc_params p;
    memcpy(&p, params, sizeof p);
    p.nthreads = 1;
    g_ops = OpCounts{};
    orc_rhs(&p, reinterpret_cast<const CD*>(gfs), reinterpret_cast<CD*>(rhs), 0, p.N[2]);
    out[0] = g_ops.add;
    out[1] = g_ops.mul;
    out[2] = g_ops.div;
    out[3] = g_ops.sqrt_;
    out[4] = g_ops.lib;
    out[5] = g_ops.cmp;
    return 0;
}
