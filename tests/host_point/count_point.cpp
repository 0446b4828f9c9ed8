// Test harness: operation census of the kernels' per-point code (bssn_point.cuh).
//
// The header is compiled for the host with every `double` replaced by a number type
// that counts the FP64 operations issued on it, and run at every interior point of a
// small grid, as k_rhs runs it for one right-hand-side evaluation (rhs_core with the
// mixed derivatives from stored first differences, then the merged advection and
// dissipation), plus the stored first differences of the k_d1 pre-pass at every point
// of its region.  The counts are those of the source: a fused multiply-add written
// fma() is one FMA, a product or a sum one multiply or add, a division one division;
// scalings by powers of two on the integer pipe (sc2) and sign flips count nothing.
// Device compilation may still contract a written product and sum into one FMA (the
// same two FLOPs) and expands the division into a reciprocal and its refinement.
#include <cmath>
#include <cstring>
#include <vector>

namespace {
struct Ops {
    long long add, mul, fma, div, sqrt_;
};
Ops g_ops;
}  // namespace

// an FP64 value whose operations are counted
struct CK {
    double v;
    constexpr CK() : v(0.0) {}
    constexpr CK(double x) : v(x) {}
    constexpr CK(int x) : v((double)x) {}
    constexpr CK(long x) : v((double)x) {}
    constexpr CK(long long x) : v((double)x) {}
    explicit operator bool() const { return v != 0.0; }
    CK& operator+=(CK b) { ++g_ops.add; v += b.v; return *this; }
    CK& operator-=(CK b) { ++g_ops.add; v -= b.v; return *this; }
    CK& operator*=(CK b) { ++g_ops.mul; v *= b.v; return *this; }
};
static_assert(sizeof(CK) == sizeof(double), "CK must be laid out as a double");
inline CK operator+(CK a, CK b) { ++g_ops.add; return CK(a.v + b.v); }
inline CK operator-(CK a, CK b) { ++g_ops.add; return CK(a.v - b.v); }
inline CK operator*(CK a, CK b) { ++g_ops.mul; return CK(a.v * b.v); }
inline CK operator/(CK a, CK b) { ++g_ops.div; return CK(a.v / b.v); }
inline CK operator-(CK a) { return CK(-a.v); }
inline bool operator<(CK a, CK b) { return a.v < b.v; }
inline bool operator>(CK a, CK b) { return a.v > b.v; }
inline bool operator<=(CK a, CK b) { return a.v <= b.v; }
inline bool operator>=(CK a, CK b) { return a.v >= b.v; }
inline bool operator==(CK a, CK b) { return a.v == b.v; }
inline bool operator!=(CK a, CK b) { return a.v != b.v; }
inline CK fma(CK a, CK b, CK c) { ++g_ops.fma; return CK(std::fma(a.v, b.v, c.v)); }
inline CK sqrt(CK a) { ++g_ops.sqrt_; return CK(std::sqrt(a.v)); }
inline CK fabs(CK a) { return CK(std::fabs(a.v)); }

// host stand-ins for the device-only names the header uses (bit manipulation: no FP64 op)
#define __device__
#define __host__
#define __forceinline__ inline
#define __global__
static inline int __double2hiint(CK x) { long long b; std::memcpy(&b, &x.v, 8); return (int)(b >> 32); }
static inline int __double2loint(CK x) { long long b; std::memcpy(&b, &x.v, 8); return (int)(b & 0xffffffffLL); }
static inline CK __hiloint2double(int hi, int lo)
{
    const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo;
    double d;
    std::memcpy(&d, &b, 8);
    return CK(d);
}
static inline long long __double_as_longlong(CK x) { long long b; std::memcpy(&b, &x.v, 8); return b; }
static inline CK __longlong_as_double(long long b) { double x; std::memcpy(&x, &b, 8); return CK(x); }
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
template <class T> static inline T __ldg(const T* p) { return *p; }

#define double CK
#include "../../paper_2505_00097_gb300/csrc/bssn_point.cuh"
#undef double
using namespace nrk;

namespace {

void radial(double A, double w, bool sinh_kind, double x, double f[4])
{
    if (sinh_kind) {
        const double s = std::sinh(1.0 / w), sh = std::sinh(x / w), ch = std::cosh(x / w);
        f[0] = A * sh / s; f[1] = A * ch / (w * s); f[2] = A * sh / (w * w * s); f[3] = A * ch / (w * w * w * s);
    } else {
        f[0] = A * x; f[1] = A; f[2] = 0.0; f[3] = 0.0;
    }
}

// counts of one right-hand-side evaluation of the interior (out[0..4]: add, mul, fma, div, sqrt)
// and of the stored first differences (out[5..9]), with the number of interior points (out[10])
// and of first-difference points (out[11]); rhs: the right-hand side (24*T doubles)
template <int FAM, int AX, int ORD>
void census(const int* N, const double* ampl, const double* sinhw, double sigma_m, double sigma_g, double eta,
            const double* y, double* rhs, long long* out)
{
    constexpr int NG = ORD / 2 + 1, E = ORD / 2;
    const bool cyl = FAM == FAM_CYL;
    int n[3];
    long T = 1;
    double lo[3], hi[3], dx[3];
    if (cyl) { lo[0] = 0; hi[0] = 1; lo[1] = -M_PI; hi[1] = M_PI; lo[2] = -1; hi[2] = 1; }
    else { lo[0] = 0; hi[0] = 1; lo[1] = 0; hi[1] = M_PI; lo[2] = -M_PI; hi[2] = M_PI; }
    for (int d = 0; d < 3; d++) { n[d] = N[d] + 2 * NG; T *= n[d]; dx[d] = (hi[d] - lo[d]) / N[d]; }
    auto xx = [&](int d, int i) { return lo[d] + ((double)(i - NG) + 0.5) * dx[d]; };
    const CK* Y = reinterpret_cast<const CK*>(y);
    // the k_d1 pre-pass region: interior i0, i1 and i2 within E of the interior except along the
    // two-point axis; the axis-1 differences at interior i1 only (general grids)
    std::vector<CK> d1x(11 * T), d1y(11 * T);
    g_ops = Ops{};
    long nd1 = 0;
    const int E1 = AX == 1 ? 0 : E, E2 = AX == 2 ? 0 : E;
    for (int i2 = NG - E2; i2 < NG + N[2] + E2; i2++)
        for (int i1 = NG - E1; i1 < NG + N[1] + E1; i1++)
            for (int i0 = NG; i0 < NG + N[0]; i0++) {
                const long idx = i0 + (long)n[0] * (i1 + (long)n[1] * i2);
                const bool ycol = AX < 0 && i1 >= NG && i1 < NG + N[1];
                for (int q = 0; q < N_D1; q++) {
                    const CK* f = Y + (long)d1gf(q) * T + idx;
                    d1x[q * T + idx] = d1r<ORD>(f, 1);
                    if (ycol) d1y[q * T + idx] = d1r<ORD>(f, n[0]);
                }
                nd1++;
            }
    const Ops d1ops = g_ops;
    g_ops = Ops{};
    double i1d[3], i2d[3];
    for (int d = 0; d < 3; d++) { i1d[d] = 1.0 / (FD<ORD>::den1.v * dx[d]); i2d[d] = 1.0 / (FD<ORD>::den2.v * dx[d] * dx[d]); }
    long nint = 0;
    for (int i2 = NG; i2 < NG + N[2]; i2++)
        for (int i1 = NG; i1 < NG + N[1]; i1++)
            for (int i0 = NG; i0 < NG + N[0]; i0++) {
                const long idx = i0 + (long)n[0] * (i1 + (long)n[1] * i2);
                PointIn P;
                P.y = Y + idx; P.T = T;
                P.st[0] = 1; P.st[1] = n[0]; P.st[2] = (long)n[0] * n[1];
                P.ox = AX == 1 ? (i1 == NG ? P.st[1] : -P.st[1]) : AX == 2 ? (i2 == NG ? P.st[2] : -P.st[2]) : 0;
                P.dx = d1x.data() + idx;
                P.dy = d1y.data() + idx;
                Geo& g = P.g;
                double f0[4];
                radial(ampl[0], sinhw[0], true, xx(0, i0), f0);
                const double s0 = 1.0 / f0[1], a = 1.0 / f0[0];
                g.a = a;
                g.d00 = f0[2] / (f0[1] * f0[1]);
                double s2;
                if (!cyl) {
                    const double th = xx(1, i1), isn = 1.0 / std::sin(th), cot = std::cos(th) / std::sin(th);
                    s2 = a * isn;
                    g.b = a; g.c = a * cot; g.d22 = 0.0;
                    g.e0a = -a * a; g.e0b = -a * a; g.e0c = -a * (a * cot); g.e1c = -s2 * s2;
                } else {
                    double fz[4];
                    radial(ampl[2], sinhw[2], true, xx(2, i2), fz);
                    s2 = 1.0 / fz[1];
                    g.d22 = fz[2] / (fz[1] * fz[1]);
                    g.b = 0.0; g.c = 0.0;
                    g.e0a = -a * a; g.e0b = 0.0; g.e0c = 0.0; g.e1c = 0.0;
                }
                const double D0 = s0 * i1d[0], D1 = a * i1d[1], D2 = s2 * i1d[2];
                g.D[0] = D0; g.D[1] = D1; g.D[2] = D2;
                g.D2[0] = s0 * s0 * i2d[0]; g.D2[1] = a * a * i2d[1]; g.D2[2] = s2 * s2 * i2d[2];
                g.DD[0] = D0 * D1; g.DD[1] = D0 * D2; g.DD[2] = D1 * D2;
                CK k[NGF];
                rhs_core<FAM, AX, true, ORD>(P, eta, k);
                add_adv_ko<AX, ORD>(P.y, T, P.st, P.ox, P.g.D, sigma_m, sigma_g, k);
                for (int q = 0; q < NGF; q++) rhs[(long)q * T + idx] = k[q].v;
                nint++;
            }
    const Ops& r = g_ops;
    const long long v[12] = {r.add, r.mul, r.fma, r.div, r.sqrt_, d1ops.add, d1ops.mul, d1ops.fma, d1ops.div,
                             d1ops.sqrt_, nint, nd1};
    for (int q = 0; q < 12; q++) out[q] = v[q];
}

// counts of the constraints at every interior point, as k_ham and k_mom run them (inline differences):
// out[0..3] add, mul, fma, div of ham_core; out[4..7] of mom_core; out[8] sqrt of mom_core; out[9] points
template <int FAM, int ORD>
void census_constraints(const int* N, const double* ampl, const double* sinhw, const double* y, long long* out)
{
    constexpr int NG = ORD / 2 + 1;
    const bool cyl = FAM == FAM_CYL;
    int n[3];
    long T = 1;
    double lo[3], hi[3], dx[3];
    if (cyl) { lo[0] = 0; hi[0] = 1; lo[1] = -M_PI; hi[1] = M_PI; lo[2] = -1; hi[2] = 1; }
    else { lo[0] = 0; hi[0] = 1; lo[1] = 0; hi[1] = M_PI; lo[2] = -M_PI; hi[2] = M_PI; }
    for (int d = 0; d < 3; d++) { n[d] = N[d] + 2 * NG; T *= n[d]; dx[d] = (hi[d] - lo[d]) / N[d]; }
    auto xx = [&](int d, int i) { return lo[d] + ((double)(i - NG) + 0.5) * dx[d]; };
    const CK* Y = reinterpret_cast<const CK*>(y);
    double i1d[3], i2d[3];
    for (int d = 0; d < 3; d++) { i1d[d] = 1.0 / (FD<ORD>::den1.v * dx[d]); i2d[d] = 1.0 / (FD<ORD>::den2.v * dx[d] * dx[d]); }
    Ops ham{}, mom{};
    long nint = 0;
    for (int i2 = NG; i2 < NG + N[2]; i2++)
        for (int i1 = NG; i1 < NG + N[1]; i1++)
            for (int i0 = NG; i0 < NG + N[0]; i0++) {
                const long idx = i0 + (long)n[0] * (i1 + (long)n[1] * i2);
                PointIn P;
                P.y = Y + idx; P.T = T;
                P.st[0] = 1; P.st[1] = n[0]; P.st[2] = (long)n[0] * n[1];
                P.ox = 0;
                P.dx = nullptr;
                P.dy = nullptr;
                Geo& g = P.g;
                double f0[4];
                radial(ampl[0], sinhw[0], true, xx(0, i0), f0);
                const double s0 = 1.0 / f0[1], a = 1.0 / f0[0];
                g.a = a;
                g.d00 = f0[2] / (f0[1] * f0[1]);
                double s2;
                if (!cyl) {
                    const double th = xx(1, i1), isn = 1.0 / std::sin(th), cot = std::cos(th) / std::sin(th);
                    s2 = a * isn;
                    g.b = a; g.c = a * cot; g.d22 = 0.0;
                    g.e0a = -a * a; g.e0b = -a * a; g.e0c = -a * (a * cot); g.e1c = -s2 * s2;
                } else {
                    double fz[4];
                    radial(ampl[2], sinhw[2], true, xx(2, i2), fz);
                    s2 = 1.0 / fz[1];
                    g.d22 = fz[2] / (fz[1] * fz[1]);
                    g.b = 0.0; g.c = 0.0;
                    g.e0a = -a * a; g.e0b = 0.0; g.e0c = 0.0; g.e1c = 0.0;
                }
                const double D0 = s0 * i1d[0], D1 = a * i1d[1], D2 = s2 * i1d[2];
                g.D[0] = D0; g.D[1] = D1; g.D[2] = D2;
                g.D2[0] = s0 * s0 * i2d[0]; g.D2[1] = a * a * i2d[1]; g.D2[2] = s2 * s2 * i2d[2];
                g.DD[0] = D0 * D1; g.DD[1] = D0 * D2; g.DD[2] = D1 * D2;
                g_ops = Ops{};
                (void)ham_core<FAM, ORD>(P);
                ham.add += g_ops.add; ham.mul += g_ops.mul; ham.fma += g_ops.fma; ham.div += g_ops.div;
                g_ops = Ops{};
                CK Mv[3];
                (void)mom_core<FAM, ORD>(P, Mv);
                mom.add += g_ops.add; mom.mul += g_ops.mul; mom.fma += g_ops.fma; mom.div += g_ops.div;
                mom.sqrt_ += g_ops.sqrt_;
                nint++;
            }
    const long long v[10] = {ham.add, ham.mul, ham.fma, ham.div, mom.add, mom.mul, mom.fma, mom.div, mom.sqrt_, nint};
    for (int q = 0; q < 10; q++) out[q] = v[q];
}

}  // namespace

// the Hamiltonian and momentum constraints' census (census_constraints), 4th or 8th order
extern "C" int census_diag(int coords, const int* N, const double* ampl, const double* sinhw, int ng, const double* y,
                           long long* out)
{
    const bool cyl = coords == 1;
    if (ng == 3) { if (cyl) census_constraints<FAM_CYL, 4>(N, ampl, sinhw, y, out); else census_constraints<FAM_SPH, 4>(N, ampl, sinhw, y, out); }
    else if (ng == 5) { if (cyl) census_constraints<FAM_CYL, 8>(N, ampl, sinhw, y, out); else census_constraints<FAM_SPH, 8>(N, ampl, sinhw, y, out); }
    else return 1;
    return 0;
}

// coords 0/2 spherical-like, 1 cylindrical-like (sinh maps on the radial and z axes); ng 3 or 5;
// the two-point specialisation where the azimuth holds two points, as the library selects it
extern "C" int census_rhs(int coords, const int* N, const double* ampl, const double* sinhw, double sigma_m,
                          double sigma_g, double eta, int ng, const double* y, double* rhs, long long* out)
{
    const bool cyl = coords == 1;
    const int ax = (cyl && N[1] == 2) ? 1 : (!cyl && N[2] == 2) ? 2 : -1;
#define CENSUS(FAM, AX, ORD) census<FAM, AX, ORD>(N, ampl, sinhw, sigma_m, sigma_g, eta, y, rhs, out)
    if (ng == 3) {
        if (cyl) { if (ax == 1) CENSUS(FAM_CYL, 1, 4); else CENSUS(FAM_CYL, -1, 4); }
        else { if (ax == 2) CENSUS(FAM_SPH, 2, 4); else CENSUS(FAM_SPH, -1, 4); }
    } else if (ng == 5) {
        if (cyl) { if (ax == 1) CENSUS(FAM_CYL, 1, 8); else CENSUS(FAM_CYL, -1, 8); }
        else { if (ax == 2) CENSUS(FAM_SPH, 2, 8); else CENSUS(FAM_SPH, -1, 8); }
    } else {
        return 1;
    }
#undef CENSUS
    return 0;
}
