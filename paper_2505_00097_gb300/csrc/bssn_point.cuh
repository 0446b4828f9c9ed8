// bssn_point.cuh -- per-point BSSN right-hand side in the orthonormal
// (rescaled) frame, FP64, for sm_103a.
//
// The evolved gridfunctions are the rescaled components of arXiv 2505.00097
// Sec. 2.2: h_ij, a_ij, lambda^i, vet^i, bet^i are the components of
// eps_ij, Abar_ij, Lambdabar^i, beta^i, B^i in the basis e~_i = e^_i / S_i,
// in which the reference metric is the identity.  This kernel evaluates the
// BSSN system of Sec. 2.1 (Eqs. metric_RHS_orig_final .. Lambda_RHS_orig_final,
// the Ricci tensor and the gauge Eqs. gauge_eqns, damping_eta_final) directly
// in that frame.  The flat reference connection Dhat then only contributes
// rotation generators with a handful of nonzero coefficients:
//   spherical-like:   Omega_1 = a J01,  Omega_2 = b J02 + c J12  (a=b=1/r, c=cot(th)/r)
//   cylindrical-like: Omega_1 = a J01                          (a=1/rho)
// where (J_pq V)_q = V_p, (J_pq V)_p = -V_q.  Only the rescaled
// gridfunctions are finite-differenced (4th-order centred; mixed second
// derivatives as products of first-derivative stencils; upwind-biased
// stencils for the beta^k d_k parts; 6th-difference Kreiss-Oliger
// dissipation), exactly as in the coordinate-basis formulation, so both give
// the same discrete right-hand side up to rounding.
//
// Readings of the paper used here: Eq. Lambda_RHS_orig_final with the two
// factors of alpha restored (-2 Abar^ij (d_j alpha - 6 alpha d_j phi) +
// 2 alpha Abar^jk Delta^i_jk); d_perp = d_t - L_beta with only the
// beta^k d_k parts upwinded; beta_j in 2 Dhat_(i beta_j) lowered with
// gammahat; Delta^k_ij built from Dhat eps only; the gauge equations with
// coordinate partial derivatives of the unrescaled beta^i, B^i, and the full
// right-hand side of Eq. Lambda_RHS_orig_final (d_perp Lambdabar^i, without the Lie
// derivative and without dissipation) inside d_t B^i.
#pragma once

#include <stdint.h>

namespace nrk {

constexpr int NGF = 24;
enum : int { G_HDD = 0, G_ADD = 6, G_CF = 12, G_TRK = 13, G_LAM = 14, G_VET = 17, G_BET = 20, G_ALPHA = 23 };
enum : int { FAM_SPH = 0, FAM_CYL = 1 };

// symmetric pair index: (0,0)=0 (0,1)=1 (0,2)=2 (1,1)=3 (1,2)=4 (2,2)=5
__host__ __device__ constexpr int sp(int i, int j) { return (i > j) ? sp(j, i) : (i == 0 ? j : (i == 1 ? j + 2 : 5)); }
__host__ __device__ constexpr int spi(int s) { return s < 3 ? 0 : (s < 5 ? 1 : 2); }
__host__ __device__ constexpr int spj(int s) { return s < 3 ? s : (s < 5 ? s - 2 : 2); }
__host__ __device__ constexpr bool offd(int s) { return s == 1 || s == 2 || s == 4; }

// Frame geometry at one point, assembled from per-axis 1D arrays.
struct Geo {
    double D[3];   // e_k f = D[k] * d1raw_k(f),  D = 1/(12 dxx_k S_k)
    double D2[3];  // 1/(12 dxx_k^2 S_k^2)
    double DD[3];  // D0 D1, D0 D2, D1 D2
    double a, b, c;                // rotation coefficients
    double d00, d22;               // dS_0/dxx0 / S_0^2, dS_2/dxx2 / S_2^2 (cylindrical)
    double e0a, e0b, e0c, e1c;     // frame derivatives of a, b, c
};

__device__ __forceinline__ double ld(const double* p) { return __ldg(p); }

// ---- raw stencil sums (weights only; spacing and scale factors in Geo)
__device__ __forceinline__ double d1raw(const double* f, long s)
{
    return fma(8.0, ld(f + s) - ld(f - s), ld(f - 2 * s) - ld(f + 2 * s));
}
__device__ __forceinline__ double d2raw(const double* f, long s)
{
    return fma(-30.0, ld(f), fma(16.0, ld(f + s) + ld(f - s), -(ld(f + 2 * s) + ld(f - 2 * s))));
}
__device__ __forceinline__ double mixraw(const double* f, long sa, long sb)
{
    double m2 = d1raw(f - 2 * sb, sa), m1 = d1raw(f - sb, sa);
    double p1 = d1raw(f + sb, sa), p2 = d1raw(f + 2 * sb, sa);
    return fma(8.0, p1 - m1, m2 - p2);
}
// upwind-biased: -3 g[-1] - 10 g[0] + 18 g[1] - 6 g[2] + g[3], g[o] = f[o*s]
// (s = -stride gives the mirrored stencil up to an overall sign)
__device__ __forceinline__ double upraw(const double* f, long s)
{
    double t1 = fma(-3.0, ld(f - s), ld(f + 3 * s));
    double t2 = fma(3.0, ld(f + s), -ld(f + 2 * s));
    return fma(-10.0, ld(f), fma(6.0, t2, t1));
}
// sixth difference without its centre term: (f-3+f3) - 6 (f-2+f2) + 15 (f-1+f1)
__device__ __forceinline__ double koraw(const double* f, long s)
{
    return fma(15.0, ld(f - s) + ld(f + s), fma(-6.0, ld(f - 2 * s) + ld(f + 2 * s), ld(f - 3 * s) + ld(f + 3 * s)));
}

// ---- 8th-order stencils (the production scheme of Sec. 4.1, N_G = 5), integer
// weights: first derivative over 840 h, second over 5040 h^2 (the scale factors
// are in Geo); a mixed derivative is the first-derivative stencil applied to the
// first differences of the neighbouring rows.
__device__ __forceinline__ double d1w8(double m4, double m3, double m2, double m1, double p1, double p2, double p3,
                                       double p4)
{
    double t = fma(-3.0, p4 - m4, 32.0 * (p3 - m3));
    t = fma(-168.0, p2 - m2, t);
    return fma(672.0, p1 - m1, t);
}
__device__ __forceinline__ double d1raw8(const double* f, long s)
{
    return d1w8(ld(f - 4 * s), ld(f - 3 * s), ld(f - 2 * s), ld(f - s), ld(f + s), ld(f + 2 * s), ld(f + 3 * s),
                ld(f + 4 * s));
}
__device__ __forceinline__ double d2raw8(const double* f, long s)
{
    double t = fma(-9.0, ld(f + 4 * s) + ld(f - 4 * s), 128.0 * (ld(f + 3 * s) + ld(f - 3 * s)));
    t = fma(-1008.0, ld(f + 2 * s) + ld(f - 2 * s), t);
    t = fma(8064.0, ld(f + s) + ld(f - s), t);
    return fma(-14350.0, ld(f), t);
}
__device__ __forceinline__ double mixraw8(const double* f, long sa, long sb)
{
    return d1w8(d1raw8(f - 4 * sb, sa), d1raw8(f - 3 * sb, sa), d1raw8(f - 2 * sb, sa), d1raw8(f - sb, sa),
                d1raw8(f + sb, sa), d1raw8(f + 2 * sb, sa), d1raw8(f + 3 * sb, sa), d1raw8(f + 4 * sb, sa));
}

// ---- scaling by 2^K: an IEEE multiply by the constant 2^K, i.e. exactly x 2^K rounded as IEEE
// specifies at every input (zeros, subnormal inputs and results, overflow to infinity, NaN).  An
// earlier version moved the exponent field on the integer pipe instead; it was faster but not the
// IEEE product at the edges of the range, and every exact integer or mixed form measured slower
// than this multiply on the head-on step.
template <int K>
__device__ __forceinline__ double sc2(double x)
{
    static_assert(K >= -60 && K <= 60, "sc2: |K| <= 60");
    constexpr auto c = K >= 0 ? 1.0 * (1ULL << (K >= 0 ? K : 0)) : 1.0 / (1ULL << (K < 0 ? -K : 0));
    return x * c;
}

// Finite-difference families: order ORD = N_FD with N_G = ORD/2 + 1 ghost layers
// (Sec. 3).  den1, den2: denominators of the integer first- and second-derivative
// weights (Geo: D = 1/(den1 dxx S), D2 = 1/(den2 dxx^2 S^2)); ko_den = 2^(2r) of
// the Kreiss-Oliger difference of order 2r = ORD + 2; ax_*: the second, upwind and
// dissipation differences along a two-point azimuth as multiples of f_other - f.
template <int ORD>
struct FD;
template <>
struct FD<4> {
    static constexpr int M = 2;
    static constexpr double den1 = 12.0, den2 = 12.0, ko_den = 64.0;
    static constexpr double ax_d2 = 32.0, ax_up = 16.0, ax_ko = 32.0;
    static constexpr int ax_d2_log2 = 5;
};
template <>
struct FD<8> {
    static constexpr int M = 4;
    static constexpr double den1 = 840.0, den2 = 5040.0, ko_den = 1024.0;
    static constexpr double ax_d2 = 16384.0, ax_up = 768.0, ax_ko = 512.0;
    static constexpr int ax_d2_log2 = 14;
};
template <int ORD>
__device__ __forceinline__ double d1r(const double* f, long s)
{
    if constexpr (ORD == 4) return d1raw(f, s);
    else return d1raw8(f, s);
}
template <int ORD>
__device__ __forceinline__ double d2r(const double* f, long s)
{
    if constexpr (ORD == 4) return d2raw(f, s);
    else return d2raw8(f, s);
}
template <int ORD>
__device__ __forceinline__ double mixr(const double* f, long sa, long sb)
{
    if constexpr (ORD == 4) return mixraw(f, sa, sb);
    else return mixraw8(f, sa, sb);
}

// ---- a periodic azimuthal axis that holds two points (AX = 1 for
// cylindrical-like, AX = 2 for spherical-like coordinates; AX = -1: none).
// Along it the neighbours at offsets +-1 and +-3 are the other slice and those
// at +-2 the point itself, so the centred first difference and every mixed
// difference that involves the axis vanish identically, and the second,
// upwind and sixth differences are 32, 16 and 32 times f_other - f (8th order:
// 16384, 768 and 512 for the second, upwind and tenth differences).  The kernels
// then skip those stencils; the result is the same discrete operator.
template <int FAM, int AX>
__host__ __device__ constexpr bool ax_ok()
{
    return AX == -1 || (FAM == FAM_CYL && AX == 1) || (FAM == FAM_SPH && AX == 2);
}
// a Hessian component known to vanish: a mixed pair that involves the axis
__host__ __device__ constexpr bool hzero(int AX, int kl) { return AX >= 0 && offd(kl) && (spi(kl) == AX || spj(kl) == AX); }
// Dhat_k V^i known to vanish: no difference along k = AX, and the generator Omega_AX never
// reaches component i (cylindrical-like: Omega_1 = a J01 leaves component 2 alone;
// spherical-like: Omega_2 = b J02 + c J12 reaches all three)
template <int FAM, int AX>
__host__ __device__ constexpr bool dvz(int i, int k)
{
    return FAM == FAM_CYL && AX == 1 && k == 1 && i == 2;
}
// Delta_ks (s = ij symmetric) known to vanish: Delta_2(12) = 1/2 Dhat_1 h_22, and on a
// cylindrical-like grid with a two-point azimuth Omega_1 h leaves the (2,2) component alone
template <int FAM, int AX>
__host__ __device__ constexpr bool dlz(int k, int s)
{
    return FAM == FAM_CYL && AX == 1 && k == 2 && s == 4;
}
// Dhat_k Dhat_l V^i known to vanish (kl symmetric index): on a cylindrical-like grid
// with a two-point azimuth, the (rho, phi) and (phi, z) pairs of component z
template <int FAM, int AX>
__host__ __device__ constexpr bool ddbz(int kl, int i)
{
    return FAM == FAM_CYL && AX == 1 && i == 2 && (kl == 1 || kl == 4);
}

// Gridfunctions with second derivatives (h, W, alpha, vet) have their raw first
// differences along axis 0 (and, for a general grid, axis 1) stored by a
// pre-pass (k_d1).  A mixed second difference is the first difference of
// those along the other axis -- the same expression mixraw evaluates -- so the
// stored path gives bitwise the result of the inline one.
constexpr int N_D1 = 11;
__host__ __device__ constexpr int d1slot(int gf)
{
    return gf < 6 ? gf : gf == G_CF ? 6 : gf == G_ALPHA ? 7 : (gf >= G_VET && gf < G_VET + 3) ? 8 + gf - G_VET : -1;
}
__host__ __device__ constexpr int d1gf(int q) { return q < 6 ? q : q == 6 ? G_CF : q == 7 ? G_ALPHA : G_VET + q - 8; }

// sum_k a_k x_k, skipping k = AX where x vanishes (AX is never 0)
template <int AX>
__device__ __forceinline__ double dot3(double a0, double a1, double a2, const double x[3])
{
    double t = a0 * x[0];
    if constexpr (AX != 1) t = fma(a1, x[1], t);
    if constexpr (AX != 2) t = fma(a2, x[2], t);
    return t;
}

// ---- frame Hessian of a component function:
// H_kl f = e_k e_l f - omega^m_kl e_m f  (symmetric in kl); ox is the offset of
// the other slice of the two-point axis
// fx, fy: stored first differences of f along axes 0 and 1 (S = true)
template <int FAM, int KL, int AX, bool S, int ORD>
__device__ __forceinline__ double hess(const double* f, const double* fx, const double* fy, const long st[3], long ox,
                                       const Geo& g, const double df[3])
{
    if constexpr (hzero(AX, KL)) return 0.0;
    if constexpr (KL == 0) return fma(g.D2[0], d2r<ORD>(f, st[0]), -g.d00 * df[0]);
    if constexpr (KL == 1) return fma(g.DD[0], S ? d1r<ORD>(fx, st[1]) : mixr<ORD>(f, st[0], st[1]), -g.a * df[1]);
    if constexpr (KL == 2) {
        const double m = S ? d1r<ORD>(fx, st[2]) : mixr<ORD>(f, st[0], st[2]);
        if constexpr (FAM == FAM_SPH) return fma(g.DD[1], m, -g.b * df[2]);
        else return g.DD[1] * m;
    }
    if constexpr (KL == 3) {
        if constexpr (AX == 1) return fma(sc2<FD<ORD>::ax_d2_log2>(g.D2[1]), ld(f + ox) - ld(f), g.a * df[0]);
        else return fma(g.D2[1], d2r<ORD>(f, st[1]), g.a * df[0]);
    }
    if constexpr (KL == 4) {
        const double m = (S && AX < 0) ? d1r<ORD>(fy, st[2]) : mixr<ORD>(f, st[1], st[2]);
        if constexpr (FAM == FAM_SPH) return fma(g.DD[2], m, -g.c * df[2]);
        else return g.DD[2] * m;
    }
    if constexpr (KL == 5) {
        if constexpr (FAM == FAM_SPH) {
            if constexpr (AX == 2)
                return fma(sc2<FD<ORD>::ax_d2_log2>(g.D2[2]), ld(f + ox) - ld(f), fma(g.b, df[0], g.c * df[1]));
            else return fma(g.D2[2], d2r<ORD>(f, st[2]), fma(g.b, df[0], g.c * df[1]));
        } else {
            return fma(g.D2[2], d2r<ORD>(f, st[2]), -g.d22 * df[2]);
        }
    }
    return 0.0;
}

template <int FAM, int AX, bool S, int ORD>
__device__ __forceinline__ void hess6(const double* f, const double* fx, const double* fy, const long st[3], long ox,
                                      const Geo& g, const double df[3], double H[6])
{
    H[0] = hess<FAM, 0, AX, S, ORD>(f, fx, fy, st, ox, g, df);
    H[1] = hess<FAM, 1, AX, S, ORD>(f, fx, fy, st, ox, g, df);
    H[2] = hess<FAM, 2, AX, S, ORD>(f, fx, fy, st, ox, g, df);
    H[3] = hess<FAM, 3, AX, S, ORD>(f, fx, fy, st, ox, g, df);
    H[4] = hess<FAM, 4, AX, S, ORD>(f, fx, fy, st, ox, g, df);
    H[5] = hess<FAM, 5, AX, S, ORD>(f, fx, fy, st, ox, g, df);
}
// gammabar^kl H_kl (gw: off-diagonal entries doubled), skipping vanishing components
template <int AX>
__device__ __forceinline__ double contract6(const double gw[6], const double H[6])
{
    double t = gw[0] * H[0];
#pragma unroll
    for (int kl = 1; kl < 6; kl++)
        if (!hzero(AX, kl)) t = fma(gw[kl], H[kl], t);
    return t;
}

// ---- rotation generators acting on vectors / symmetric tensors: out += c * J_pq (.)
__device__ __forceinline__ void j01v(double c, const double V[3], double o[3]) { o[1] = fma(c, V[0], o[1]); o[0] = fma(-c, V[1], o[0]); }
__device__ __forceinline__ void j02v(double c, const double V[3], double o[3]) { o[2] = fma(c, V[0], o[2]); o[0] = fma(-c, V[2], o[0]); }
__device__ __forceinline__ void j12v(double c, const double V[3], double o[3]) { o[2] = fma(c, V[1], o[2]); o[1] = fma(-c, V[2], o[1]); }

__device__ __forceinline__ void j01s(double c, const double T[6], double o[6])
{
    const double c2 = sc2<1>(c);
    o[0] = fma(-c2, T[1], o[0]);
    o[1] = fma(c, T[0] - T[3], o[1]);
    o[2] = fma(-c, T[4], o[2]);
    o[3] = fma(c2, T[1], o[3]);
    o[4] = fma(c, T[2], o[4]);
}
__device__ __forceinline__ void j02s(double c, const double T[6], double o[6])
{
    const double c2 = sc2<1>(c);
    o[0] = fma(-c2, T[2], o[0]);
    o[1] = fma(-c, T[4], o[1]);
    o[2] = fma(c, T[0] - T[5], o[2]);
    o[4] = fma(c, T[1], o[4]);
    o[5] = fma(c2, T[2], o[5]);
}
__device__ __forceinline__ void j12s(double c, const double T[6], double o[6])
{
    const double c2 = sc2<1>(c);
    o[1] = fma(-c, T[2], o[1]);
    o[2] = fma(c, T[1], o[2]);
    o[3] = fma(-c2, T[4], o[3]);
    o[4] = fma(c, T[3] - T[5], o[4]);
    o[5] = fma(c2, T[4], o[5]);
}

// Omega_k acting on a vector / symmetric tensor, accumulated into o
template <int FAM, int K>
__device__ __forceinline__ void omv(const Geo& g, double s, const double V[3], double o[3])
{
    if constexpr (K == 1) j01v(g.a * s, V, o);
    if constexpr (K == 2 && FAM == FAM_SPH) { j02v(g.b * s, V, o); j12v(g.c * s, V, o); }
}
template <int FAM, int K>
__device__ __forceinline__ void oms(const Geo& g, double s, const double T[6], double o[6])
{
    if constexpr (K == 1) j01s(g.a * s, T, o);
    if constexpr (K == 2 && FAM == FAM_SPH) { j02s(g.b * s, T, o); j12s(g.c * s, T, o); }
}

__device__ __forceinline__ double gsym(const double m[6], int i, int j) { return m[sp(i, j)]; }

// Inputs of the point evaluation that the kernel precomputes once.
struct PointIn {
    const double* y;  // state at this point: y + idx (gridfunction g at y[g*T])
    long T;
    long st[3];
    long ox;          // offset of the other slice of a two-point azimuthal axis (unused otherwise)
    // stored raw first differences d1raw along axis 0 (dx) and axis 1 (dy) of the
    // gridfunctions with second derivatives, at this point (slot q at dx[q*T]);
    // NULL where the kernel differences inline
    const double* dx;
    const double* dy;
    Geo g;
};

// e_k of gridfunction gf: zero along the two-point axis, from the stored first
// differences where the point has them (S), else inline
template <int AX, bool S, int ORD>
__device__ __forceinline__ double der1(const PointIn& P, int gf, int k)
{
    if (k == AX) return 0.0;
    const int q = d1slot(gf);
    if (S && q >= 0 && k == 0) return P.g.D[0] * ld(P.dx + (long)q * P.T);
    if (S && AX < 0 && q >= 0 && k == 1) return P.g.D[1] * ld(P.dy + (long)q * P.T);
    return P.g.D[k] * d1r<ORD>(P.y + (long)gf * P.T, P.st[k]);
}
template <bool S>
__device__ __forceinline__ const double* dxp(const PointIn& P, int gf)
{
    return S ? P.dx + (long)d1slot(gf) * P.T : nullptr;
}
template <int AX, bool S>
__device__ __forceinline__ const double* dyp(const PointIn& P, int gf)
{
    return (S && AX < 0) ? P.dy + (long)d1slot(gf) * P.T : nullptr;
}

// Metric-sector quantities shared by the right-hand side and the
// Hamiltonian constraint.
struct MetricPart {
    double h[6], gi[6], gw[6];
    double dh[3][6];
    double GH[6];        // gammabar^ij H_kl h_ij
    double Dl[3][6];     // Delta_kij (first index lowered)
    double Dup[3][6];    // Delta^k_ij
    double Dvec[3];      // Delta^k
    double Dtr[3];       // Delta^k_km
    double Ric[6];       // Rbar_ij
    double W, iW, dphi[3];
    double DDphir[6];    // Dbar_i Dbar_j phi - 2 e_i phi e_j phi (what every consumer needs)
};

// The conformal metric and its inverse, first frame derivatives of h, and
// Delta (lowered, raised, its trace Delta^k and Delta^k_km): shared by the
// right-hand side and both constraints.
template <int FAM, int AX, bool S, int ORD>
__device__ __forceinline__ void metric_first(const PointIn& P, MetricPart& M)
{
    static_assert(ax_ok<FAM, AX>(), "two-point axis must be the azimuth");
    const double* y = P.y;
    const long T = P.T;
    const Geo& g = P.g;
    auto F = [&](int gf) { return y + (long)gf * T; };
    double* h = M.h;
    double* gi = M.gi;
    double* gw = M.gw;
#pragma unroll
    for (int s = 0; s < 6; s++) h[s] = ld(F(G_HDD + s));
    const double W = ld(F(G_CF));
    M.W = W;

    // ---------------- conformal metric gammabar_ij = delta_ij + h_ij and its inverse
    const double g00 = 1.0 + h[0], g11 = 1.0 + h[3], g22 = 1.0 + h[5];
    gi[0] = fma(g11, g22, -h[4] * h[4]);
    gi[1] = fma(h[2], h[4], -h[1] * g22);
    gi[2] = fma(h[1], h[4], -h[2] * g11);
    gi[3] = fma(g00, g22, -h[2] * h[2]);
    gi[4] = fma(h[1], h[2], -g00 * h[4]);
    gi[5] = fma(g00, g11, -h[1] * h[1]);
    const double det = fma(g00, gi[0], fma(h[1], gi[1], h[2] * gi[2]));
    const double rdw = 1.0 / (det * W);   // one division gives 1/det and 1/W
    const double idet = rdw * W;
    M.iW = rdw * det;
#pragma unroll
    for (int s = 0; s < 6; s++) gi[s] *= idet;
#pragma unroll
    for (int s = 0; s < 6; s++) gw[s] = offd(s) ? sc2<1>(gi[s]) : gi[s];

    // ---------------- first frame derivatives of h
    double (*dh)[6] = M.dh;
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int s = 0; s < 6; s++) dh[k][s] = der1<AX, S, ORD>(P, G_HDD + s, k);

    // ---------------- Dhat_k h_ij, Delta_kij (first index lowered), Delta^k_ij, Delta^k
    double Dh[3][6];
#pragma unroll
    for (int s = 0; s < 6; s++) { Dh[0][s] = dh[0][s]; Dh[1][s] = dh[1][s]; Dh[2][s] = dh[2][s]; }
    oms<FAM, 1>(g, 1.0, h, Dh[1]);
    oms<FAM, 2>(g, 1.0, h, Dh[2]);
    double (*Dl)[6] = M.Dl;
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const int i = spi(s), j = spj(s);
            // Delta_kij = 1/2 (Dhat_i h_jk + Dhat_j h_ik - Dhat_k h_ij); with k = j (k = i) the
            // last two (the first and last) terms are the same number and cancel exactly
            if (k == j)
                Dl[k][s] = sc2<-1>(Dh[i][sp(k, k)]);
            else if (k == i)
                Dl[k][s] = sc2<-1>(Dh[j][sp(k, k)]);
            else
                Dl[k][s] = sc2<-1>(Dh[i][sp(j, k)] + Dh[j][sp(i, k)] - Dh[k][s]);
        }
    double (*Dup)[6] = M.Dup;
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int s = 0; s < 6; s++) {
            double t = fma(gsym(gi, k, 1), Dl[1][s], gsym(gi, k, 0) * Dl[0][s]);
            Dup[k][s] = dlz<FAM, AX>(2, s) ? t : fma(gsym(gi, k, 2), Dl[2][s], t);
        }
    double* Dvec = M.Dvec;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double t = gw[0] * Dup[k][0];
#pragma unroll
        for (int s = 1; s < 6; s++) t = fma(gw[s], Dup[k][s], t);
        Dvec[k] = t;
    }
    // Delta^k_km = 1/2 gammabar^ab e_m h_ab
#pragma unroll
    for (int m = 0; m < 3; m++) {
        double t = gw[0] * dh[m][0];
#pragma unroll
        for (int s = 1; s < 6; s++) t = fma(gw[s], dh[m][s], t);
        M.Dtr[m] = m == AX ? 0.0 : sc2<-1>(t);
    }
}

template <int FAM, bool NEED_GH, int AX, bool S, int ORD>
__device__ __forceinline__ void metric_part(const PointIn& P, MetricPart& M)
{
    metric_first<FAM, AX, S, ORD>(P, M);
    const double* y = P.y;
    const long T = P.T;
    const Geo& g = P.g;
    const long* st = P.st;
    auto F = [&](int gf) { return y + (long)gf * T; };
    const double* h = M.h;
    const double* gi = M.gi;
    const double* gw = M.gw;
    const double (*dh)[6] = M.dh;
    const double (*Dl)[6] = M.Dl;
    const double (*Dup)[6] = M.Dup;
    const double* Dvec = M.Dvec;

    // ---------------- Hessians of h contracted two ways:
    // Lh_ij = gammabar^kl H_kl h_ij,  GH_kl = gammabar^ij H_kl h_ij
    double Lh[6];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        double df[3] = {dh[0][s], dh[1][s], dh[2][s]};
        double H[6];
        hess6<FAM, AX, S, ORD>(F(G_HDD + s), dxp<S>(P, G_HDD + s), dyp<AX, S>(P, G_HDD + s), st, P.ox, g, df, H);
        Lh[s] = contract6<AX>(gw, H);
        if constexpr (NEED_GH) {
#pragma unroll
            for (int kl = 0; kl < 6; kl++) {
                if (hzero(AX, kl)) M.GH[kl] = 0.0;
                else M.GH[kl] = s == 0 ? gw[0] * H[kl] : fma(gw[s], H[kl], M.GH[kl]);
            }
        }
    }

    // ---------------- Ricci tensor
    // gammabar^kl Dhat_k Dhat_l h_ij = Lh + 2 Omega_l.V_l + (linear and quadratic generator terms).h
    double Lfull[6];
    {
        double V1[6], V2[6], Y1[6] = {0, 0, 0, 0, 0, 0}, Y2[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const double d[3] = {dh[0][s], dh[1][s], dh[2][s]};
            V1[s] = dot3<AX>(gi[1], gi[3], gi[4], d);
            V2[s] = dot3<AX>(gi[2], gi[4], gi[5], d);
        }
        j01s(g.a, h, Y1);                                                        // Y1 = Omega_1 h
        if constexpr (FAM == FAM_SPH) { j02s(g.b, h, Y2); j12s(g.c, h, Y2); }    // Y2 = Omega_2 h
        double X01[6], X02[6], X12[6];
        const double a2 = sc2<1>(g.a);
        if constexpr (FAM == FAM_SPH) {
            const double c1 = fma(g.a, gi[1], -g.c * gi[5]);
            const double c2 = fma(g.b, gi[2], g.c * gi[4]);
            const double g01 = fma(gi[1], g.e0a, -c1 * g.a);
            const double g02 = fma(gi[2], g.e0b, -c2 * g.b);
            const double g12 = fma(gi[2], g.e0c, fma(gi[4], g.e1c, -c2 * g.c));
            const double b2 = sc2<1>(g.b), cc2 = sc2<1>(g.c);
            const double a11 = g.a * gi[3], a12 = g.a * gi[4];
            const double b12 = g.b * gi[4], b22 = g.b * gi[5];
            const double k12 = g.c * gi[4], k22 = g.c * gi[5];
#pragma unroll
            for (int s = 0; s < 6; s++) {
                X01[s] = fma(a2, V1[s], fma(g01, h[s], fma(a11, Y1[s], a12 * Y2[s])));
                // (Omega_1 h)_22 = 0; X01's (2,2) component is never read
                X02[s] = fma(b2, V2[s], fma(g02, h[s], s == 5 ? b22 * Y2[s] : fma(b12, Y1[s], b22 * Y2[s])));
                X12[s] = fma(cc2, V2[s], fma(g12, h[s], s == 5 ? k22 * Y2[s] : fma(k12, Y1[s], k22 * Y2[s])));
            }
        } else {
            const double g01 = gi[1] * (g.e0a - g.a * g.a);
            const double a11 = g.a * gi[3];
#pragma unroll
            for (int s = 0; s < 6; s++) X01[s] = fma(a2, V1[s], fma(g01, h[s], a11 * Y1[s]));
        }
#pragma unroll
        for (int s = 0; s < 6; s++) Lfull[s] = Lh[s];
        j01s(1.0, X01, Lfull);
        if constexpr (FAM == FAM_SPH) { j02s(1.0, X02, Lfull); j12s(1.0, X12, Lfull); }
    }
    // Dhat_j lambda^k
    double lam[3], Dlam[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++) lam[i] = ld(F(G_LAM + i));
#pragma unroll
    for (int j = 0; j < 3; j++)
#pragma unroll
        for (int k = 0; k < 3; k++) Dlam[j][k] = der1<AX, S, ORD>(P, G_LAM + k, j);
    omv<FAM, 1>(g, 1.0, lam, Dlam[1]);
    omv<FAM, 2>(g, 1.0, lam, Dlam[2]);
    // Quadratic terms. With R[i][m][l] = gammabar^lk Delta^m_ik,
    //   gammabar^kl Delta^m_ki Delta_jml = sum_ml R[i][m][l] Delta_jml   (A_ij; Delta_jml is
    //                                      symmetric in ml, so R is summed over the pair first)
    //   gammabar^kl Delta^m_ik Delta_mjl = sum_ml R[i][m][l] Delta_mjl   (C_ij, symmetric)
    // and R_ij = -1/2 Lfull_ij + A_ij + A_ji + C_ij + 1/2 (Lambda and Delta^k terms), each
    // component one chain with the 1/2 taken into the factors.
    double R[3][3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int m = 0; m < 3; m++)
#pragma unroll
            for (int l = 0; l < 3; l++)
                R[i][m][l] = fma(Dup[m][sp(2, i)], gsym(gi, 2, l),
                                 fma(Dup[m][sp(1, i)], gsym(gi, 1, l), Dup[m][sp(0, i)] * gsym(gi, 0, l)));
    double Rp[3][6];   // Rp[i][p] = R[i][m][l] + R[i][l][m] for the pair p = (m, l), R[i][m][m] on the diagonal
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int p = 0; p < 6; p++) Rp[i][p] = offd(p) ? R[i][spi(p)][spj(p)] + R[i][spj(p)][spi(p)] : R[i][spi(p)][spi(p)];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const int i = spi(s), j = spj(s);
        // C_ij
        double t = R[i][0][0] * Dl[0][sp(j, 0)];
#pragma unroll
        for (int q = 1; q < 9; q++) {
            const int m = q / 3, l = q % 3;
            if (!dlz<FAM, AX>(m, sp(j, l))) t = fma(R[i][m][l], Dl[m][sp(j, l)], t);
        }
        // (Dl[k][p] = 0 where dlz(k, p) and Dlam[j][k] = Dhat_j lambda^k = 0 where dvz(k, j):
        // those terms are skipped)
        if (i == j) {
            // 2 A_ii (A_ii summed on its own, doubled by the FMA that adds it)
            double u = 0.0;
#pragma unroll
            for (int p = 0; p < 6; p++)
                if (!dlz<FAM, AX>(i, p)) u = fma(Rp[i][p], Dl[i][p], u);
            t = fma(2.0, u, t);
            // 1/2 Delta^k (2 Delta_iik)
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (!dlz<FAM, AX>(i, sp(i, k))) t = fma(Dvec[k], Dl[i][sp(i, k)], t);
            // 1/2 (2 gammabar_ki Dhat_i lambda^k)
            if (!dvz<FAM, AX>(i, i)) t += Dlam[i][i];
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (!dvz<FAM, AX>(k, i)) t = fma(h[sp(k, i)], Dlam[i][k], t);
        } else {
            // A_ij + A_ji
#pragma unroll
            for (int p = 0; p < 6; p++)
                if (!dlz<FAM, AX>(j, p)) t = fma(Rp[i][p], Dl[j][p], t);
#pragma unroll
            for (int p = 0; p < 6; p++)
                if (!dlz<FAM, AX>(i, p)) t = fma(Rp[j][p], Dl[i][p], t);
            // 1/2 Delta^k (Delta_ijk + Delta_jik) + 1/2 (gammabar_ki Dhat_j lambda^k + gammabar_kj
            // Dhat_i lambda^k): summed on their own, halved by the FMA that adds them
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (!dlz<FAM, AX>(i, sp(j, k))) v = fma(Dvec[k], Dl[i][sp(j, k)], v);
                if (!dlz<FAM, AX>(j, sp(i, k))) v = fma(Dvec[k], Dl[j][sp(i, k)], v);
            }
            if (!dvz<FAM, AX>(i, j)) v += Dlam[j][i];
            if (!dvz<FAM, AX>(j, i)) v += Dlam[i][j];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (!dvz<FAM, AX>(k, i)) v = fma(h[sp(k, j)], Dlam[i][k], v);
                if (!dvz<FAM, AX>(k, j)) v = fma(h[sp(k, i)], Dlam[j][k], v);
            }
            t = fma(0.5, v, t);
        }
        M.Ric[s] = fma(-0.5, Lfull[s], t);
    }

    // ---------------- conformal factor: phi = -1/2 ln W
    double dW[3];
#pragma unroll
    for (int k = 0; k < 3; k++) dW[k] = der1<AX, S, ORD>(P, G_CF, k);
    const double mhiW = -sc2<-1>(M.iW);
#pragma unroll
    for (int k = 0; k < 3; k++) M.dphi[k] = k == AX ? 0.0 : mhiW * dW[k];
    {
        double HW[6];
        hess6<FAM, AX, S, ORD>(F(G_CF), dxp<S>(P, G_CF), dyp<AX, S>(P, G_CF), st, P.ox, g, dW, HW);
#pragma unroll
        for (int s = 0; s < 6; s++) {
            // e_i e_j phi = -1/2 W^-1 H_ij W + 2 e_i phi e_j phi; the second term is left out
            const double dd = dot3<AX>(Dup[0][s], Dup[1][s], Dup[2][s], M.dphi);
            M.DDphir[s] = hzero(AX, s) ? -dd : fma(mhiW, HW[s], -dd);
        }
    }
}

// Output: the 24 right-hand sides without the beta^k d_k advection and
// without Kreiss-Oliger dissipation (added by the caller, see adv_ko()).
template <int FAM, int AX, bool S, int ORD>
__device__ __forceinline__ void rhs_core(const PointIn& P, double eta, double out[NGF])
{
    const double* y = P.y;
    const long T = P.T;
    const Geo& g = P.g;
    const long* st = P.st;
    auto F = [&](int gf) { return y + (long)gf * T; };

    MetricPart M;
    metric_part<FAM, true, AX, S, ORD>(P, M);
    const double* h = M.h;
    const double* gi = M.gi;
    const double* gw = M.gw;
    const double (*dh)[6] = M.dh;
    const double (*Dup)[6] = M.Dup;
    const double* Dvec = M.Dvec;
    const double* Dtr = M.Dtr;
    const double* GH = M.GH;
    const double* Ric = M.Ric;
    const double* dphi = M.dphi;
    const double* DDphir = M.DDphir;
    const double W = M.W;

    double a[6], lam[3], vet[3], bet[3];
#pragma unroll
    for (int s = 0; s < 6; s++) a[s] = ld(F(G_ADD + s));
#pragma unroll
    for (int i = 0; i < 3; i++) { lam[i] = ld(F(G_LAM + i)); vet[i] = ld(F(G_VET + i)); bet[i] = ld(F(G_BET + i)); }
    const double K = ld(F(G_TRK)), al = ld(F(G_ALPHA));
    const double al2 = sc2<1>(al);   // 2 alpha
    double dK[3], dal[3], dvet[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        dK[k] = der1<AX, S, ORD>(P, G_TRK, k);
        dal[k] = der1<AX, S, ORD>(P, G_ALPHA, k);
#pragma unroll
        for (int i = 0; i < 3; i++) dvet[k][i] = der1<AX, S, ORD>(P, G_VET + i, k);
    }
    double DDal[6];
    {
        double Hal[6];
        hess6<FAM, AX, S, ORD>(F(G_ALPHA), dxp<S>(P, G_ALPHA), dyp<AX, S>(P, G_ALPHA), st, P.ox, g, dal, Hal);
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const double dd = dot3<AX>(Dup[0][s], Dup[1][s], Dup[2][s], dal);
            DDal[s] = hzero(AX, s) ? -dd : Hal[s] - dd;
        }
    }

    // ---------------- Abar with raised indices
    double Aud[3][3];  // Abar^k_j
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            Aud[k][j] = fma(gsym(gi, k, 2), a[sp(2, j)], fma(gsym(gi, k, 1), a[sp(1, j)], gsym(gi, k, 0) * a[sp(0, j)]));
    double Auu[6];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const int i = spi(s), j = spj(s);
        Auu[s] = fma(Aud[i][2], gsym(gi, 2, j), fma(Aud[i][1], gsym(gi, 1, j), Aud[i][0] * gsym(gi, 0, j)));
    }
    const double trA = Aud[0][0] + Aud[1][1] + Aud[2][2];
    double AA = a[0] * Auu[0];
#pragma unroll
    for (int s = 1; s < 6; s++) AA = fma(offd(s) ? sc2<1>(a[s]) : a[s], Auu[s], AA);

    // ---------------- shift: Dhat_k beta^i, second covariant derivatives, divergences
    double Db[3][3];  // Db[i][k] = Dhat_k beta^i
    {
        // the generator terms accumulate onto the differences (no additions of zeros)
        double c1[3] = {dvet[1][0], dvet[1][1], dvet[1][2]}, c2[3] = {dvet[2][0], dvet[2][1], dvet[2][2]};
        omv<FAM, 1>(g, 1.0, vet, c1);
        omv<FAM, 2>(g, 1.0, vet, c2);
#pragma unroll
        for (int i = 0; i < 3; i++) { Db[i][0] = dvet[0][i]; Db[i][1] = c1[i]; Db[i][2] = c2[i]; }
    }
    const double divhat = Db[0][0] + Db[1][1] + Db[2][2];
    double divbar = divhat;
#pragma unroll
    for (int m = 0; m < 3; m++)
        if (m != AX) divbar = fma(Dtr[m], vet[m], divbar);
    // DDb[kl][i] = Dhat_k Dhat_l beta^i
    double DDb[6][3];
    {
        double Hv[3][6];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            double df[3] = {dvet[0][i], dvet[1][i], dvet[2][i]};
            hess6<FAM, AX, S, ORD>(F(G_VET + i), dxp<S>(P, G_VET + i), dyp<AX, S>(P, G_VET + i), st, P.ox, g, df,
                              Hv[i]);
        }
#pragma unroll
        for (int kl = 0; kl < 6; kl++)
#pragma unroll
            for (int i = 0; i < 3; i++) DDb[kl][i] = Hv[i][kl];
        // (0,1): J01 (a e_0 vet + e0a vet)
        {
            double t[3];
#pragma unroll
            for (int i = 0; i < 3; i++) t[i] = fma(g.a, dvet[0][i], g.e0a * vet[i]);
            j01v(1.0, t, DDb[1]);
        }
        // (1,1): J01 (2 a e_1 vet + a^2 J01 vet)
        {
            double u[3] = {0, 0, 0};
            j01v(g.a * g.a, vet, u);
            double t[3];
            const double a2 = sc2<1>(g.a);
#pragma unroll
            for (int i = 0; i < 3; i++) t[i] = AX == 1 ? u[i] : fma(a2, dvet[1][i], u[i]);   // e_1 vet = 0 on AX = 1
            j01v(1.0, t, DDb[3]);
        }
        if constexpr (FAM == FAM_SPH) {
            // (0,2): J02 (b e_0 vet + e0b vet) + J12 (c e_0 vet + e0c vet)
            {
                double t[3], u[3];
#pragma unroll
                for (int i = 0; i < 3; i++) { t[i] = fma(g.b, dvet[0][i], g.e0b * vet[i]); u[i] = fma(g.c, dvet[0][i], g.e0c * vet[i]); }
                j02v(1.0, t, DDb[2]);
                j12v(1.0, u, DDb[2]);
            }
            // Z = Omega_2 vet
            double Z[3] = {0, 0, 0};
            j02v(g.b, vet, Z);
            j12v(g.c, vet, Z);
            // (1,2): J02 (b e_1 vet) + J12 (c e_1 vet + e1c vet) + J01 (a e_2 vet + a Z)
            {
                double t[3], u[3], w[3];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    t[i] = g.b * dvet[1][i];
                    u[i] = fma(g.c, dvet[1][i], g.e1c * vet[i]);
                    w[i] = g.a * (dvet[2][i] + Z[i]);
                }
                j02v(1.0, t, DDb[4]);
                j12v(1.0, u, DDb[4]);
                j01v(1.0, w, DDb[4]);
            }
            // (2,2): J01 (c a vet) + J02 (2 b e_2 vet + b Z) + J12 (2 c e_2 vet + c Z)
            {
                double t[3], u[3];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const double e2 = sc2<1>(dvet[2][i]);
                    t[i] = g.b * (e2 + Z[i]);
                    u[i] = g.c * (e2 + Z[i]);
                }
                j01v(g.c * g.a, vet, DDb[5]);
                j02v(1.0, t, DDb[5]);
                j12v(1.0, u, DDb[5]);
            }
        } else {
            // (1,2): J01 (a e_2 vet)
            double w[3];
#pragma unroll
            for (int i = 0; i < 3; i++) w[i] = g.a * dvet[2][i];
            j01v(1.0, w, DDb[4]);
        }
    }
    // gammabar^kl Dhat_k Dhat_l beta^i
    double LapB[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double t = gw[0] * DDb[0][i];
#pragma unroll
        for (int kl = 1; kl < 6; kl++)
            if (!ddbz<FAM, AX>(kl, i)) t = fma(gw[kl], DDb[kl][i], t);
        LapB[i] = t;
    }
    // e_l (Dbar_k beta^k) = sum_k DDb[kl][k] + sum_m [e_l(Delta^k_km) vet^m + Delta^k_km e_l vet^m]
    // e_l(Delta^k_km) = 1/2 (GH_lm - Q_lm) - (Omega_l Dtr)_m,  Q_lm = tr(gbinv e_l h gbinv e_m h)
    double gdiv[3];
    {
        double M[3][3][3];  // M[l] = gbinv . e_l h  (zero along the two-point axis)
#pragma unroll
        for (int l = 0; l < 3; l++)
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++)
                    M[l][i][j] = l == AX ? 0.0 : fma(gsym(gi, i, 2), dh[l][sp(2, j)], fma(gsym(gi, i, 1), dh[l][sp(1, j)], gsym(gi, i, 0) * dh[l][sp(0, j)]));
        double Q[6];
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const int l = spi(s), m = spj(s);
            if (l == AX || m == AX) {
                Q[s] = 0.0;
                continue;
            }
            double t = M[l][0][0] * M[m][0][0];
#pragma unroll
            for (int q = 1; q < 9; q++) t = fma(M[l][q / 3][q % 3], M[m][q % 3][q / 3], t);
            Q[s] = t;
        }
        double OD[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // (Omega_l Dtr)
        omv<FAM, 1>(g, 1.0, Dtr, OD[1]);
        omv<FAM, 2>(g, 1.0, Dtr, OD[2]);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            double t = DDb[sp(l, 0)][0] + DDb[sp(l, 1)][1];
            if (!ddbz<FAM, AX>(sp(l, 2), 2)) t += DDb[sp(l, 2)][2];
#pragma unroll
            for (int m = 0; m < 3; m++) {
                // with exactly one of l, m on the two-point axis, GH, Q and (Omega_l Dtr)_m all
                // vanish; Dtr[AX] = 0 and e_AX vet = 0
                if (l != AX && m != AX) t = fma(Dtr[m], dvet[l][m], t);
                if (AX < 0 || (l == AX) == (m == AX)) {
                    const double edtr = fma(0.5, GH[sp(l, m)] - Q[sp(l, m)], -OD[l][m]);
                    t = fma(edtr, vet[m], t);
                }
            }
            gdiv[l] = t;
        }
    }

    // ================= right-hand sides (advection and dissipation excluded)
    // Eq. metric_RHS_orig_final + Lie terms:
    // d_t h_ij = [Omega part of beta^k Dhat_k h_ij] + gammabar_kj Dhat_i beta^k + gammabar_ik Dhat_j beta^k
    //            - 2/3 gammabar_ij (Dbar.beta - alpha Abar^k_k) - 2 alpha a_ij
    {
        double r[6];
        const double tt = (2.0 / 3.0) * fma(-al, trA, divbar);
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const int i = spi(s), j = spj(s);
            // (Db[k][i] = 0 where dvz(k, i): those terms are skipped)
            const bool zji = dvz<FAM, AX>(j, i), zij = dvz<FAM, AX>(i, j);
            double t = zji ? (zij ? 0.0 : Db[i][j]) : (zij ? Db[j][i] : Db[j][i] + Db[i][j]);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (!dvz<FAM, AX>(k, j)) t = fma(h[sp(i, k)], Db[k][j], t);
                if (!dvz<FAM, AX>(k, i)) t = fma(h[sp(k, j)], Db[k][i], t);
            }
            const double gij = (i == j) ? 1.0 + h[s] : h[s];
            r[s] = fma(-al2, a[s], fma(-tt, gij, t));
        }
        oms<FAM, 1>(g, vet[1], h, r);
        oms<FAM, 2>(g, vet[2], h, r);
#pragma unroll
        for (int s = 0; s < 6; s++) out[G_HDD + s] = r[s];
    }
    // Eq. Abar_RHS_orig_final + Lie terms
    {
        double X[6];
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const int i = spi(s), j = spj(s);
            // 2 alpha (2 e_i phi e_j phi - Dbar_i Dbar_j phi) = -2 alpha DDphir, and
            // 2 (e_i alpha e_j phi + e_j alpha e_i phi), which vanishes when i or j is the
            // two-point axis
            double t = fma(-al2, DDphir[s], -DDal[s]);
            if (i != AX && j != AX)
                t = i == j ? fma(sc2<2>(dal[i]), dphi[i], t)
                           : fma(sc2<1>(dal[i]), dphi[j], fma(sc2<1>(dal[j]), dphi[i], t));
            X[s] = fma(al, Ric[s], t);
        }
        double trX = gw[0] * X[0];
#pragma unroll
        for (int s = 1; s < 6; s++) trX = fma(gw[s], X[s], trX);
        const double W2 = W * W;
        const double third_trX = trX * (1.0 / 3.0);
        const double c_div = (-2.0 / 3.0) * divbar + al * K;
        double r[6];
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const int i = spi(s), j = spj(s);
            double t = fma(a[sp(0, j)], Db[0][i], a[sp(i, 0)] * Db[0][j]);
#pragma unroll
            for (int k = 1; k < 3; k++) {
                if (!dvz<FAM, AX>(k, j)) t = fma(a[sp(i, k)], Db[k][j], t);
                if (!dvz<FAM, AX>(k, i)) t = fma(a[sp(k, j)], Db[k][i], t);
            }
            const double AAij = fma(a[sp(i, 2)], Aud[2][j], fma(a[sp(i, 1)], Aud[1][j], a[sp(i, 0)] * Aud[0][j]));
            const double gij = (i == j) ? 1.0 + h[s] : h[s];
            const double XTF = fma(-third_trX, gij, X[s]);
            r[s] = fma(W2, XTF, fma(-al2, AAij, fma(c_div, a[s], t)));
        }
        oms<FAM, 1>(g, vet[1], a, r);
        oms<FAM, 2>(g, vet[2], a, r);
#pragma unroll
        for (int s = 0; s < 6; s++) out[G_ADD + s] = r[s];
        // Eq. W_RHS_orig_final
        out[G_CF] = (-1.0 / 3.0) * W * fma(-al, K, divbar);
        // Eq. K_RHS_orig_final
        double lapal = gw[0] * DDal[0], gap = gw[0] * dal[0] * dphi[0];
#pragma unroll
        for (int s = 1; s < 6; s++) {
            const int i = spi(s), j = spj(s);
            lapal = fma(gw[s], DDal[s], lapal);
            if (i == AX || j == AX) continue;   // d_AX alpha = d_AX phi = 0
            gap = fma(gi[s], (i == j) ? dal[i] * dphi[i] : fma(dal[i], dphi[j], dal[j] * dphi[i]), gap);
        }
        out[G_TRK] = fma(al, fma((1.0 / 3.0) * K, K, AA), -W2 * fma(2.0, gap, lapal));
    }
    // Eq. Lambda_RHS_orig_final (with the alpha factors restored) + Lie terms
    double rl[3], rperp[3];
    {
        // wl_j = -2 (d_j alpha - 6 alpha d_j phi); zero along the two-point axis
        double wl[3];
        const double al12 = 12.0 * al;
#pragma unroll
        for (int k = 0; k < 3; k++) wl[k] = k == AX ? 0.0 : fma(al12, dphi[k], -sc2<1>(dal[k]));
#pragma unroll
        for (int i = 0; i < 3; i++) {
            // (2/3) Delta^i Dbar.beta + (1/3) gammabar^ik e_k Dbar.beta (the Lie-derivative part
            // - lambda^j Dhat_j beta^i + beta^j (Omega_j lambda)^i is added after this block)
            double t = LapB[i];
            t = fma((2.0 / 3.0) * Dvec[i], divbar, t);
            t = fma((1.0 / 3.0), fma(gsym(gi, i, 2), gdiv[2], fma(gsym(gi, i, 1), gdiv[1], gsym(gi, i, 0) * gdiv[0])), t);
            // -2 Abar^ij (d_j alpha - 6 alpha d_j phi) - 4/3 alpha gammabar^ij d_j K
            const double v = dot3<AX>(gsym(gi, i, 0), gsym(gi, i, 1), gsym(gi, i, 2), dK);
            t = fma((-4.0 / 3.0) * al, v, t);
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k != AX) t = fma(Auu[sp(i, k)], wl[k], t);
            // + 2 alpha Abar^jk Delta^i_jk
            double w = Auu[0] * Dup[i][0];
#pragma unroll
            for (int s = 1; s < 6; s++) w = fma(offd(s) ? sc2<1>(Auu[s]) : Auu[s], Dup[i][s], w);
            rl[i] = fma(al2, w, t);
        }
        // Lie-derivative part: - lambda^j Dhat_j beta^i + beta^j (Omega_j lambda)^i
#pragma unroll
        for (int i = 0; i < 3; i++) rperp[i] = rl[i];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            double t = fma(-lam[0], Db[i][0], rl[i]);
            if (!dvz<FAM, AX>(i, 1)) t = fma(-lam[1], Db[i][1], t);
            rl[i] = fma(-lam[2], Db[i][2], t);
        }
        omv<FAM, 1>(g, vet[1], lam, rl);
        omv<FAM, 2>(g, vet[2], lam, rl);
#pragma unroll
        for (int i = 0; i < 3; i++) out[G_LAM + i] = rl[i];
    }
    // gauge: d_t alpha = -2 alpha K (+ advection);  d_t beta^i = B^i (+ coordinate advection);
    //        d_t B^i = 3/4 [right-hand side of Eq. Lambda, i.e. d_perp Lambdabar^i] - eta B^i
    //                  (+ coordinate advection)
    {
        // partial-derivative advection of unrescaled components: - v^i sum_j d_ij vet^j
        double dv[3];
        dv[0] = g.d00 * vet[0];
        dv[1] = g.a * vet[0];
        if constexpr (FAM == FAM_SPH) dv[2] = fma(g.b, vet[0], g.c * vet[1]);
        else dv[2] = g.d22 * vet[2];
        out[G_ALPHA] = -al2 * K;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            out[G_VET + i] = fma(-vet[i], dv[i], bet[i]);
            out[G_BET + i] = fma(-bet[i], dv[i], fma(0.75, rperp[i], -eta * bet[i]));
        }
    }
}

// Hamiltonian constraint, Eq. Hconstraint:
// H = 2/3 K^2 - Abar_ij Abar^ij + W^2 (Rbar - 8 gammabar^ij d_i phi d_j phi - 8 gammabar^ij Dbar_i Dbar_j phi)
template <int FAM, int ORD>
__device__ __forceinline__ double ham_core(const PointIn& P)
{
    MetricPart M;
    metric_part<FAM, false, -1, false, ORD>(P, M);
    const double* gi = M.gi;
    const double* gw = M.gw;
    double a[6];
#pragma unroll
    for (int s = 0; s < 6; s++) a[s] = ld(P.y + (long)(G_ADD + s) * P.T);
    const double K = ld(P.y + (long)G_TRK * P.T);
    double Aud[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            Aud[k][j] = fma(gsym(gi, k, 2), a[sp(2, j)], fma(gsym(gi, k, 1), a[sp(1, j)], gsym(gi, k, 0) * a[sp(0, j)]));
    // Abar_ij Abar^ij = Abar^i_j Abar^j_i
    double AA = Aud[0][0] * Aud[0][0];
#pragma unroll
    for (int q = 1; q < 9; q++) AA = fma(Aud[q / 3][q % 3], Aud[q % 3][q / 3], AA);
    // gammabar^ij (Dbar_i Dbar_j phi + e_i phi e_j phi) = lp + 3 gp with lp over DDphir
    double R = gw[0] * M.Ric[0], gp = gw[0] * M.dphi[0] * M.dphi[0], lp = gw[0] * M.DDphir[0];
#pragma unroll
    for (int s = 1; s < 6; s++) {
        R = fma(gw[s], M.Ric[s], R);
        gp = fma(gw[s], M.dphi[spi(s)] * M.dphi[spj(s)], gp);
        lp = fma(gw[s], M.DDphir[s], lp);
    }
    return fma((2.0 / 3.0) * K, K, fma(M.W * M.W, fma(-8.0, fma(3.0, gp, lp), R), -AA));
}

// Momentum constraint, Eq. Mconstraint.  Its first two terms are Dbar_j Abar^ij
// (Dhat_j Abar^ij + Delta^i_jk Abar^kj + Delta^j_jk Abar^ik), evaluated here
// with metric compatibility as gammabar^ik gammabar^jl Dbar_j Abar_kl and
// Dbar_j Abar_kl = Dhat_j Abar_kl - Delta^m_jk Abar_ml - Delta^m_jl Abar_km:
//   M^i = W^2 (gammabar^ik V_k + 6 Abar^ij e_j phi - 2/3 gammabar^ij e_j K),
//   V_k = gammabar^jl Dhat_j a_kl - Delta^m_jk Abar^j_m - a_km Delta^m.
// Writes the frame (rescaled) components M^i; returns |M| = sqrt(gamma_ij M^i M^j)
// with the physical metric gamma_ij = gammabar_ij / W^2.
template <int FAM, int ORD>
__device__ __forceinline__ double mom_core(const PointIn& P, double Mv[3])
{
    MetricPart M;
    metric_first<FAM, -1, false, ORD>(P, M);
    const double* y = P.y;
    const long T = P.T;
    const Geo& g = P.g;
    const long* st = P.st;
    auto F = [&](int gf) { return y + (long)gf * T; };
    const double* gi = M.gi;
    const double (*Dup)[6] = M.Dup;
    const double W = M.W;
    double a[6], Da[3][6], dK[3], dphi[3];
#pragma unroll
    for (int s = 0; s < 6; s++) a[s] = ld(F(G_ADD + s));
#pragma unroll
    for (int k = 0; k < 3; k++) {
#pragma unroll
        for (int s = 0; s < 6; s++) Da[k][s] = g.D[k] * d1r<ORD>(F(G_ADD + s), st[k]);
        dK[k] = g.D[k] * d1r<ORD>(F(G_TRK), st[k]);
        dphi[k] = (-0.5 * M.iW) * (g.D[k] * d1r<ORD>(F(G_CF), st[k]));
    }
    oms<FAM, 1>(g, 1.0, a, Da[1]);   // Dhat_k a_ij
    oms<FAM, 2>(g, 1.0, a, Da[2]);
    double Aud[3][3];  // Abar^k_j
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            Aud[k][j] = fma(gsym(gi, k, 2), a[sp(2, j)], fma(gsym(gi, k, 1), a[sp(1, j)], gsym(gi, k, 0) * a[sp(0, j)]));
    double V[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int l = 0; l < 3; l++) t = fma(gsym(gi, j, l), Da[j][sp(k, l)], t);
#pragma unroll
        for (int j = 0; j < 3; j++)
#pragma unroll
            for (int m = 0; m < 3; m++) t = fma(-Dup[m][sp(j, k)], Aud[j][m], t);
#pragma unroll
        for (int m = 0; m < 3; m++) t = fma(-a[sp(k, m)], M.Dvec[m], t);
        V[k] = t;
    }
    const double W2 = W * W;
    double q = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            // Abar^ij = Abar^i_k gammabar^kj
            const double Auu = fma(Aud[i][2], gsym(gi, 2, j), fma(Aud[i][1], gsym(gi, 1, j), Aud[i][0] * gsym(gi, 0, j)));
            t = fma(gsym(gi, i, j), fma((-2.0 / 3.0), dK[j], V[j]), fma(6.0 * Auu, dphi[j], t));
        }
        Mv[i] = W2 * t;
    }
    // gamma_ij M^i M^j = (M.M + h_ij M^i M^j) / W^2
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const int i = spi(s), j = spj(s);
        const double hm = (offd(s) ? 2.0 : 1.0) * M.h[s] * Mv[i] * Mv[j];
        q += (i == j) ? fma(Mv[i], Mv[i], hm) : hm;
    }
    return sqrt(q) * M.iW;
}

// beta^k d_k f, upwinded, and the Kreiss-Oliger dissipation of f, evaluated as
// one 7-point stencil per axis whose weights are formed once per point.  Along
// axis k, with u = |vet^k| D_k (D_k = 1/(12 dxx_k S_k)), p = u, q = 0 for
// vet^k > 0 (upwind offsets -1..+3) and p = 0, q = u otherwise (offsets
// -3..+1), and kap = sigma/(64 S_k dxx_k) = (12/64) sigma D_k (the strength
// refers to the physical spacing), the weights at offsets -3..+3 are
//   q+kap, -6(q+kap), 18q-3p+15kap, -10u-20kap, 18p-3q+15kap, -6(p+kap), p+kap,
// i.e. u times the upwind weights (-3,-10,18,-6,1)/(12 dxx_k S_k) on the side
// of vet^k, plus kap times the sixth difference (1,-6,15,-20,15,-6,1).  Along
// a two-point axis the sum is (16u + 32kap)(f_other - f).
struct AdvKoW {
    double w[3][6];   // per axis: offsets -3, -2, -1, +1, +2, +3
    double c0;        // centre weight summed over the axes (with -cax folded in)
    double cax;       // two-point axis: weight of f_other (the sum along it is cax (f_other - f))
};

template <int AX>
__device__ __forceinline__ void advko_weights(const double u[3], const bool fwd[3], const double D[3], double sigma,
                                              AdvKoW& W)
{
    double c0 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double kap = (0.1875 * sigma) * D[d];
        if (d == AX) {
            W.cax = fma(16.0, u[d], sc2<5>(kap));   // FD<4>::ax_up u + FD<4>::ax_ko kap
            continue;
        }
        const double p = fwd[d] ? u[d] : 0.0, q = fwd[d] ? 0.0 : u[d];
        const double pk = p + kap, qk = q + kap, k15 = 15.0 * kap;
        W.w[d][0] = qk;
        W.w[d][1] = -6.0 * qk;
        W.w[d][2] = fma(18.0, q, fma(-3.0, p, k15));
        W.w[d][3] = fma(18.0, p, fma(-3.0, q, k15));
        W.w[d][4] = -6.0 * pk;
        W.w[d][5] = pk;
        c0 = d == 0 ? fma(-10.0, u[d], -20.0 * kap) : c0 + fma(-10.0, u[d], -20.0 * kap);
    }
    W.c0 = AX >= 0 ? c0 - W.cax : c0;
}

template <int AX>
__device__ __forceinline__ double advko_apply(const double* f, const long st[3], long ox, const AdvKoW& W, double k)
{
    k = fma(W.c0, ld(f), k);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d == AX) {
            k = fma(W.cax, ld(f + ox), k);
            continue;
        }
        const long s = st[d];
        k = fma(W.w[d][0], ld(f - 3 * s), k);
        k = fma(W.w[d][1], ld(f - 2 * s), k);
        k = fma(W.w[d][2], ld(f - s), k);
        k = fma(W.w[d][3], ld(f + s), k);
        k = fma(W.w[d][4], ld(f + 2 * s), k);
        k = fma(W.w[d][5], ld(f + 3 * s), k);
    }
    return k;
}

// 8th order: upwind weights on offsets -3..+5 (over 840; the backward stencil
// uses them mirrored) and the tenth difference on -5..+5, as one 11-point
// stencil per axis.  Along a two-point azimuth the sum is
// (768 u + 512 kap)(f_other - f), kap = sigma/(1024 S_k dxx_k) = (840/1024) sigma D_k.
__host__ __device__ constexpr double up8(int o)
{
    return o == -3 ? -5.0 : o == -2 ? 60.0 : o == -1 ? -420.0 : o == 0 ? -378.0 : o == 1 ? 1050.0
         : o == 2 ? -420.0 : o == 3 ? 140.0 : o == 4 ? -30.0 : o == 5 ? 3.0 : 0.0;
}
__host__ __device__ constexpr double ko10(int o)
{
    return o == 0 ? -252.0 : (o == 1 || o == -1) ? 210.0 : (o == 2 || o == -2) ? -120.0
         : (o == 3 || o == -3) ? 45.0 : (o == 4 || o == -4) ? -10.0 : (o == 5 || o == -5) ? 1.0 : 0.0;
}
__host__ __device__ constexpr int off10(int j) { return j < 5 ? j - 5 : j - 4; }   // offsets -5..-1, 1..5

struct AdvKoW8 {
    double w[3][10];   // per axis, offsets off10(j)
    double c0;         // centre weight summed over the axes (with -cax folded in)
    double cax;        // two-point axis: weight of f_other (the sum along it is cax (f_other - f))
};

template <int AX>
__device__ __forceinline__ void advko_weights8(const double u[3], const bool fwd[3], const double D[3], double sigma,
                                               AdvKoW8& W)
{
    double c0 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double kap = (0.8203125 * sigma) * D[d];
        if (d == AX) {
            W.cax = fma(768.0, u[d], sc2<9>(kap));  // FD<8>::ax_up u + FD<8>::ax_ko kap
            continue;
        }
        const double p = fwd[d] ? u[d] : 0.0, q = fwd[d] ? 0.0 : u[d];
#pragma unroll
        for (int j = 0; j < 10; j++) {
            const int o = off10(j);
            double w = ko10(o) * kap;
            if (up8(o) != 0.0) w = fma(p, up8(o), w);
            if (up8(-o) != 0.0) w = fma(q, up8(-o), w);
            W.w[d][j] = w;
        }
        const double c = fma(-378.0, u[d], -252.0 * kap);   // p + q = u
        c0 = d == 0 ? c : c0 + c;
    }
    W.c0 = AX >= 0 ? c0 - W.cax : c0;
}

template <int AX>
__device__ __forceinline__ double advko_apply8(const double* f, const long st[3], long ox, const AdvKoW8& W, double k)
{
    k = fma(W.c0, ld(f), k);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d == AX) {
            k = fma(W.cax, ld(f + ox), k);
            continue;
        }
#pragma unroll
        for (int j = 0; j < 10; j++) k = fma(W.w[d][j], ld(f + off10(j) * st[d]), k);
    }
    return k;
}

// Adds the upwinded advection and the dissipation to the 24 right-hand sides
// of rhs_core: sigma_metric on the 17 metric gridfunctions (h, a, W, K,
// lambda), sigma_gauge on the 7 gauge gridfunctions (vet, bet, alpha).
template <int AX, int ORD>
__device__ __forceinline__ void add_adv_ko(const double* y, long T, const long st[3], long ox, const double D[3],
                                           double sigma_metric, double sigma_gauge, double k[NGF])
{
    double u[3];
    bool fwd[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double v = ld(y + (long)(G_VET + d) * T);
        u[d] = fabs(v) * D[d];
        // v > 0 by the sign of the bit pattern, on the integer pipe: the same answer for
        // every value but NaN (+0 and -0 both give the backward stencil)
        fwd[d] = __double_as_longlong(v) > 0;
    }
    if constexpr (ORD == 8) {
        AdvKoW8 Wm, Wg;
        advko_weights8<AX>(u, fwd, D, sigma_metric, Wm);
        advko_weights8<AX>(u, fwd, D, sigma_gauge, Wg);
#pragma unroll
        for (int g = 0; g < NGF; g++) k[g] = advko_apply8<AX>(y + (long)g * T, st, ox, g < G_VET ? Wm : Wg, k[g]);
    } else {
        AdvKoW Wm, Wg;
        advko_weights<AX>(u, fwd, D, sigma_metric, Wm);
        advko_weights<AX>(u, fwd, D, sigma_gauge, Wg);
#pragma unroll
        for (int g = 0; g < NGF; g++) k[g] = advko_apply<AX>(y + (long)g * T, st, ox, g < G_VET ? Wm : Wg, k[g]);
    }
}

}  // namespace nrk
