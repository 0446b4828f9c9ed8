// Test harness: the per-point BSSN math of the CUDA kernels (bssn_point.cuh), compiled for
// the host with g++, evaluated at every interior point of a small grid.  It lets the CPU
// test suite compare the kernels' arithmetic with the oracle without a GPU.  The grid
// geometry below follows the same definitions as the library's set-up (Sec. 2.2: the
// rescaling factors of SinhSpherical, SinhCylindrical and Spherical coordinates and their
// first and second derivatives), restated here so the harness needs nothing but the
// per-point header.
#include <cmath>
#include <cstring>
#include <vector>

// host stand-ins for the device-only names the header uses
#define __device__
#define __host__
#define __forceinline__ inline
#define __global__
static inline int __double2hiint(double x) { long long b; std::memcpy(&b, &x, 8); return (int)(b >> 32); }
static inline int __double2loint(double x) { long long b; std::memcpy(&b, &x, 8); return (int)(b & 0xffffffffLL); }
static inline double __hiloint2double(int hi, int lo)
{
    const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo;
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}
static inline long long __double_as_longlong(double x) { long long b; std::memcpy(&b, &x, 8); return b; }
static inline double __longlong_as_double(long long b) { double x; std::memcpy(&x, &b, 8); return x; }
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
template <class T> static inline T __ldg(const T* p) { return *p; }
using std::fma;

#include "../../paper_2505_00097_gb300/csrc/bssn_point.cuh"
using namespace nrk;

namespace {

// x -> (A sinh(x/w)/sinh(1/w)) and its first three derivatives; linear (A x) without sinh
void radial(double A, double w, bool sinh_kind, double x, double f[4])
{
    if (sinh_kind) {
        const double s = std::sinh(1.0 / w), sh = std::sinh(x / w), ch = std::cosh(x / w);
        f[0] = A * sh / s; f[1] = A * ch / (w * s); f[2] = A * sh / (w * w * s); f[3] = A * ch / (w * w * w * s);
    } else {
        f[0] = A * x; f[1] = A; f[2] = 0.0; f[3] = 0.0;
    }
}

template <int FAM, int AX, int ORD>
void point_rhs(PointIn& P, bool S, double eta, const double* sigma, long T, double k[NGF])
{
    if (S) rhs_core<FAM, AX, true, ORD>(P, eta, k);
    else rhs_core<FAM, AX, false, ORD>(P, eta, k);
    add_adv_ko<AX, ORD>(P.y, T, P.st, P.ox, P.g.D, sigma[0], sigma[G_VET], k);
}

template <int ORD>
void host_point_t(int coords, const int* N, const double* ampl, const double* sinhw, const double* sigma, double eta,
                  const double* y, double* out, int which)
{
    const int NG = ORD / 2 + 1;
    const bool cyl = coords == 1;
    int n[3];
    long T = 1;
    double lo[3], hi[3], dx[3];
    if (cyl) { lo[0] = 0; hi[0] = 1; lo[1] = -M_PI; hi[1] = M_PI; lo[2] = -1; hi[2] = 1; }
    else { lo[0] = 0; hi[0] = 1; lo[1] = 0; hi[1] = M_PI; lo[2] = -M_PI; hi[2] = M_PI; }
    for (int d = 0; d < 3; d++) { n[d] = N[d] + 2 * NG; T *= n[d]; dx[d] = (hi[d] - lo[d]) / N[d]; }
    auto xx = [&](int d, int i) { return lo[d] + ((double)(i - NG) + 0.5) * dx[d]; };
    double i1d[3], i2d[3];
    for (int d = 0; d < 3; d++) { i1d[d] = 1.0 / (FD<ORD>::den1 * dx[d]); i2d[d] = 1.0 / (FD<ORD>::den2 * dx[d] * dx[d]); }

    // stored raw first differences along axes 0 and 1 (the k_d1 pre-pass), where asked for
    std::vector<double> d1x(11 * T, 0.0), d1y(11 * T, 0.0);
    if (which == 3) {
        for (int i2 = NG - ORD / 2; i2 < NG + N[2] + ORD / 2; i2++)
            for (int i1 = NG - ORD / 2; i1 < NG + N[1] + ORD / 2; i1++)
                for (int i0 = NG; i0 < NG + N[0]; i0++) {
                    const long idx = i0 + (long)n[0] * (i1 + (long)n[1] * i2);
                    for (int q = 0; q < 11; q++) {
                        const double* f = y + (long)d1gf(q) * T + idx;
                        d1x[q * T + idx] = d1r<ORD>(f, 1);
                        if (i1 >= ORD / 2 && i1 < n[1] - ORD / 2) d1y[q * T + idx] = d1r<ORD>(f, n[0]);
                    }
                }
    }
    const int ax = (cyl && N[1] == 2) ? 1 : (!cyl && N[2] == 2) ? 2 : -1;
    for (int i2 = NG; i2 < NG + N[2]; i2++)
        for (int i1 = NG; i1 < NG + N[1]; i1++)
            for (int i0 = NG; i0 < NG + N[0]; i0++) {
                const long idx = i0 + (long)n[0] * (i1 + (long)n[1] * i2);
                PointIn P;
                P.y = y + idx; P.T = T;
                P.st[0] = 1; P.st[1] = n[0]; P.st[2] = (long)n[0] * n[1];
                P.dx = nullptr; P.dy = nullptr; P.ox = 0;
                Geo& g = P.g;
                double f0[4];
                radial(ampl[0], sinhw[0], coords != 2, xx(0, i0), f0);
                const double s0 = 1.0 / f0[1], a = 1.0 / f0[0];
                g.a = a;
                g.d00 = f0[2] / (f0[1] * f0[1]);
                double s2;
                if (!cyl) {
                    const double th = xx(1, i1), isn = 1.0 / std::sin(th), cot = std::cos(th) / std::sin(th);
                    s2 = a * isn;
                    g.b = a; g.c = a * cot; g.d22 = 0.0;
                    g.e0a = -a * a; g.e0b = g.e0a; g.e0c = -a * g.c; g.e1c = -s2 * s2;
                } else {
                    double fz[4];
                    radial(ampl[2], sinhw[2], true, xx(2, i2), fz);
                    s2 = 1.0 / fz[1];
                    g.d22 = fz[2] / (fz[1] * fz[1]);
                    g.b = g.c = 0.0;
                    g.e0a = -a * a; g.e0b = g.e0c = g.e1c = 0.0;
                }
                g.D[0] = s0 * i1d[0]; g.D[1] = a * i1d[1]; g.D[2] = s2 * i1d[2];
                g.D2[0] = s0 * s0 * i2d[0]; g.D2[1] = a * a * i2d[1]; g.D2[2] = s2 * s2 * i2d[2];
                g.DD[0] = g.D[0] * g.D[1]; g.DD[1] = g.D[0] * g.D[2]; g.DD[2] = g.D[1] * g.D[2];
                if (which == 1) {
                    out[idx] = cyl ? ham_core<FAM_CYL, ORD>(P) : ham_core<FAM_SPH, ORD>(P);
                    continue;
                }
                if (which == 2) {
                    double Mv[3];
                    if (cyl) mom_core<FAM_CYL, ORD>(P, Mv); else mom_core<FAM_SPH, ORD>(P, Mv);
                    for (int q = 0; q < 3; q++) out[(long)q * T + idx] = Mv[q];
                    continue;
                }
                if (ax == 1) P.ox = i1 == NG ? P.st[1] : -P.st[1];
                else if (ax == 2) P.ox = i2 == NG ? P.st[2] : -P.st[2];
                P.dx = d1x.data() + idx;
                P.dy = d1y.data() + idx;
                const bool S = which == 3;
                double k[NGF];
                if (!cyl) {
                    if (ax == 2) point_rhs<FAM_SPH, 2, ORD>(P, S, eta, sigma, T, k);
                    else point_rhs<FAM_SPH, -1, ORD>(P, S, eta, sigma, T, k);
                } else {
                    if (ax == 1) point_rhs<FAM_CYL, 1, ORD>(P, S, eta, sigma, T, k);
                    else point_rhs<FAM_CYL, -1, ORD>(P, S, eta, sigma, T, k);
                }
                for (int q = 0; q < NGF; q++) out[(long)q * T + idx] = k[q];
            }
}

}  // namespace

// which: 0 the RHS (rhs_core + advection + dissipation) with inline differences, 3 the same
// from stored first differences, 1 the Hamiltonian constraint, 2 the momentum constraint.
// sigma: the dissipation strength per gridfunction (metric at 0, gauge at G_VET).
extern "C" void host_point(int coords, const int* N, const double* ampl, const double* sinhw, const double* sigma,
                           double eta, const double* y, double* out, int which, int ng)
{
    if (ng == 5) host_point_t<8>(coords, N, ampl, sinhw, sigma, eta, y, out, which);
    else host_point_t<4>(coords, N, ampl, sinhw, sigma, eta, y, out, which);
}

// the exact power-of-two scaling of the point code, sc2<K>, for the K it uses
extern "C" int host_sc2(int K, const double* x, double* out, long n)
{
    for (long i = 0; i < n; i++) {
        switch (K) {
        case -1: out[i] = sc2<-1>(x[i]); break;
        case 1: out[i] = sc2<1>(x[i]); break;
        case 2: out[i] = sc2<2>(x[i]); break;
        case 5: out[i] = sc2<5>(x[i]); break;
        case 9: out[i] = sc2<9>(x[i]); break;
        default: return 1;
        }
    }
    return 0;
}
