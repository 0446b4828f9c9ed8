// nr_stage.cuh -- per-point bodies of the RK4-stage kernels, shared by the
// single-grid kernels (nr_kernels.cu) and the batched kernel
// (nr_batch.cu) so that both run bit-identical arithmetic per point.
#pragma once

#include "bssn_point.cuh"
#include "nr_geo.cuh"
#include "nr_internal.h"

namespace nrk {

// det(delta_ij + h_ij) := 1 (Lagrangian choice of Sec. 2.1), in place, in
// terms of the deviation h so that small h keeps its relative precision:
// f(x) = (1 + x)^(-1/3) - 1.  After every substage |x| = |det - 1| is small: there the
// binomial series to x^6 (C(-1/3, k): -1/3, 2/9, -14/81, 35/243, -91/729, 728/6561) in
// Horner form; for |x| <= 2^-10 the first omitted term, |C(-1/3, 7)| x^7 ~ 0.1 x^7, is below
// 3e-19 |f|, far under an ulp.  Elsewhere f = expm1(-log1p(x)/3).  f(0) = 0 exactly.
__device__ __forceinline__ double rcbrt1p_m1(double x)
{
    // |x| <= 2^-10 by the magnitude bits, on the integer pipe (NaN takes the other branch)
    if ((unsigned long long)(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL) <= 0x3F50000000000000ULL) {
        double p = fma(728.0 / 6561.0, x, -91.0 / 729.0);
        p = fma(p, x, 35.0 / 243.0);
        p = fma(p, x, -14.0 / 81.0);
        p = fma(p, x, 2.0 / 9.0);
        p = fma(p, x, -1.0 / 3.0);
        return p * x;
    }
    return expm1(log1p(x) * (-1.0 / 3.0));
}

// det(I + h) - 1 = tr h + (sum of principal 2x2 minors of h) + det h,
// f1 = det^(-1/3) - 1, h <- h + f1 (delta + h).
__device__ __forceinline__ void enforce_det(double* v)
{
    const double m2 = fma(v[0], v[3], fma(v[0], v[5], fma(v[3], v[5], -fma(v[1], v[1], fma(v[2], v[2], v[4] * v[4])))));
    const double c0 = fma(v[3], v[5], -v[4] * v[4]);
    const double c1 = fma(v[2], v[4], -v[1] * v[5]);
    const double c2 = fma(v[1], v[4], -v[2] * v[3]);
    const double d3 = fma(v[0], c0, fma(v[1], c1, v[2] * c2));
    const double dm1 = (v[0] + v[3] + v[5]) + (m2 + d3);
    const double f1 = rcbrt1p_m1(dm1);
    v[0] = fma(f1, v[0], v[0] + f1);
    v[1] = fma(f1, v[1], v[1]);
    v[2] = fma(f1, v[2], v[2]);
    v[3] = fma(f1, v[3], v[3] + f1);
    v[4] = fma(f1, v[4], v[4]);
    v[5] = fma(f1, v[5], v[5] + f1);
}

// Whether the first SSPRK3 stage takes the short form y + dt k in stage_store (the general form
// with its zero and unit weights gives the same numbers but for the sign of a zero): measured
// 0.8 % faster per step in the two-point-azimuth kernels, 1.6 % slower in the general 8th-order
// kernel on a 384x192x384 grid, whose register allocation it changes
template <int AX>
__host__ __device__ constexpr bool ssp_first_short()
{
    return AX >= 0;
}

// Stage epilogue for one point: k -> (y_next, acc), or the plain RHS.  yin: the
// stage input (read by MODE_SSP at this point).  yn may equal out (the last
// SSPRK3 stage updates y_n in place: each point reads its own values first).
template <bool SHORT1>
__device__ __forceinline__ void stage_store(const Stage& st, long T, long idx, const double k[NGF],
                                            const double* yin, const double* yn, double* out,
                                            double* __restrict__ acc)
{
    if (st.mode == MODE_RHS) {
#pragma unroll
        for (int g = 0; g < NGF; g++) out[g * T + idx] = k[g];
        return;
    }
    double v[NGF];
    if (st.mode == MODE_SSP) {
        if (SHORT1 && st.cyn == 0.0 && st.cacc == 1.0) {
            // the first stage, y_1 = y + dt k: the general form's 0 y_n + 1 (.) left out
#pragma unroll
            for (int g = 0; g < NGF; g++) v[g] = fma(st.cnext, k[g], yin[g * T + idx]);
        } else {
#pragma unroll
            for (int g = 0; g < NGF; g++)
                v[g] = fma(st.cyn, yn[g * T + idx], st.cacc * fma(st.cnext, k[g], yin[g * T + idx]));
        }
    } else if (st.mode == MODE_STAGE4) {
#pragma unroll
        for (int g = 0; g < NGF; g++) v[g] = fma(st.cacc, k[g], acc[g * T + idx]);
    } else {
        // every load ahead of the first store: the offsets g T are run-time values, so a store to
        // acc may alias a later load of acc as far as the compiler can tell, and a load-update-store
        // loop would wait out one memory latency per gridfunction (measured: 10 % of the launch)
        double a[NGF];
#pragma unroll
        for (int g = 0; g < NGF; g++) {
            v[g] = yn[g * T + idx];
            a[g] = st.mode == MODE_STAGE1 ? v[g] : acc[g * T + idx];
        }
#pragma unroll
        for (int g = 0; g < NGF; g++) {
            acc[g * T + idx] = fma(st.cacc, k[g], a[g]);
            v[g] = fma(st.cnext, k[g], v[g]);
        }
    }
    if (st.enforce) enforce_det(v);
#pragma unroll
    for (int g = 0; g < NGF; g++) out[g * T + idx] = v[g];
    if (st.mirror) {
        const long r = st.rank[idx];
#pragma unroll
        for (int g = 0; g < NGF; g++) st.mirror[g * st.mirror_n + r] = v[g];
    }
}

// one-sided / centred first-derivative stencil sums (weights of 12 h f')
__device__ __forceinline__ double osraw(const double* f, long s, int kind)
{
    switch (kind) {
    case 0: return fma(8.0, ld(f + s) - ld(f - s), ld(f - 2 * s) - ld(f + 2 * s));
    case 1: return fma(3.0, ld(f + s), fma(10.0, ld(f), fma(-18.0, ld(f - s), fma(6.0, ld(f - 2 * s), -ld(f - 3 * s)))));
    case 2: return fma(25.0, ld(f), fma(-48.0, ld(f - s), fma(36.0, ld(f - 2 * s), fma(-16.0, ld(f - 3 * s), 3.0 * ld(f - 4 * s)))));
    case 3: return fma(-3.0, ld(f - s), fma(-10.0, ld(f), fma(18.0, ld(f + s), fma(-6.0, ld(f + 2 * s), ld(f + 3 * s)))));
    default: return fma(-25.0, ld(f), fma(48.0, ld(f + s), fma(-36.0, ld(f + 2 * s), fma(16.0, ld(f + 3 * s), -3.0 * ld(f + 4 * s)))));
    }
}

// 8th-order one-sided first derivative on the window a..a+8, a = -w (w = 0..8),
// integer weights over 840 h; w = 4 is the centred stencil
__host__ __device__ constexpr double os8(int w, int i)
{
    constexpr double t[9][9] = {
        {-2283, 6720, -11760, 15680, -14700, 9408, -3920, 960, -105},
        {-105, -1338, 2940, -2940, 2450, -1470, 588, -140, 15},
        {15, -240, -798, 1680, -1050, 560, -210, 48, -5},
        {-5, 60, -420, -378, 1050, -420, 140, -30, 3},
        {3, -32, 168, -672, 0, 672, -168, 32, -3},
        {-3, 30, -140, 420, -1050, 378, 420, -60, 5},
        {5, -48, 210, -560, 1050, -1680, 798, 240, -15},
        {-15, 140, -588, 1470, -2450, 2940, -2940, 1338, 105},
        {105, -960, 3920, -9408, 14700, -15680, 11760, -6720, 2283}};
    return t[w][i];
}
__device__ __forceinline__ double osraw8(const double* f, long s, int w)
{
    double t = 0.0;
    switch (w) {
#define OS8_CASE(W)                                                                         \
    case W:                                                                                 \
        _Pragma("unroll") for (int i = 0; i < 9; i++) t = fma(os8(W, i), ld(f + (i - W) * s), t); \
        return t;
        OS8_CASE(0) OS8_CASE(1) OS8_CASE(2) OS8_CASE(3) OS8_CASE(4) OS8_CASE(5) OS8_CASE(6) OS8_CASE(7)
        OS8_CASE(8)
#undef OS8_CASE
    default: return 0.0;
    }
}

__device__ __forceinline__ int gf_type(int g)
{
    if (g < 6) return 4 + g;
    if (g < 12) return g - 2;
    if (g == G_CF || g == G_TRK || g == G_ALPHA) return 0;
    if (g < G_VET) return g - G_LAM + 1;
    if (g < G_BET) return g - G_VET + 1;
    return g - G_BET + 1;
}

// one interior point (interior-relative i in [0,N0), j = i1 + N1 i2 in [0, N1 N2)) of an RK stage:
// right-hand side, upwinded advection, dissipation and the stage epilogue.  AX: the azimuthal axis
// when it holds two points (G.ax), else -1.  S: the raw first differences along axes 0 and 1 of the
// gridfunctions with second derivatives are read from d1x, d1y (N_D1 sets of T doubles; d1y only
// for AX = -1), as k_d1 stored them from yin; the result is bitwise the same either way.
template <int FAM, int AX, bool S, int ORD>
__device__ __forceinline__ void rhs_point_stage(const GridK& G, const double* __restrict__ yin,
                                                const double* __restrict__ d1x, const double* __restrict__ d1y,
                                                double* out, const double* yn, double* acc, const Stage& st, int i,
                                                int j)
{
    const int p0 = i + G.NG, p1 = j % G.N1 + G.NG, p2 = j / G.N1 + G.NG;
    const long idx = p0 + (long)G.n0 * (p1 + (long)G.n1 * p2);
    PointIn P;
    P.y = yin + idx;
    P.T = G.T;
    P.st[0] = 1;
    P.st[1] = G.n0;
    P.st[2] = (long)G.n0 * G.n1;
    if constexpr (AX == 1) P.ox = p1 == G.NG ? P.st[1] : -P.st[1];
    else if constexpr (AX == 2) P.ox = p2 == G.NG ? P.st[2] : -P.st[2];
    else P.ox = 0;
    P.dx = S ? d1x + idx : nullptr;
    P.dy = (S && AX < 0) ? d1y + idx : nullptr;
    P.g = make_geo<FAM>(G, p0, p1, p2);
    double k[NGF];
    rhs_core<FAM, AX, S, ORD>(P, G.eta, k);
    add_adv_ko<AX, ORD>(P.y, G.T, P.st, P.ox, P.g.D, G.sigma_metric, G.sigma_gauge, k);
    stage_store<ssp_first_short<AX>()>(st, G.T, idx, k, yin, yn, out, acc);
}

// Points of the stored first differences (k_d1): interior i0, and i1 and i2 within
// two points of the interior except along a two-point azimuth, which has no mixed
// derivatives; the axis-1 set is taken at interior i1 only (general grids).
__host__ __device__ inline long d1_points(const GridK& G)
{
    const int E = G.ord / 2, E1 = G.ax == 1 ? 0 : E, E2 = G.ax == 2 ? 0 : E;
    return (long)G.N0 * (G.N1 + 2 * E1) * (G.N2 + 2 * E2);
}

// point t of that region: raw first differences along axis 0 (and 1) of the N_D1
// gridfunctions with second derivatives
template <int AX, int ORD>
__device__ __forceinline__ void d1_point(const GridK& G, const double* __restrict__ y, double* d1x, double* d1y, long t)
{
    constexpr int E1 = AX == 1 ? 0 : ORD / 2, E2 = AX == 2 ? 0 : ORD / 2;
    const int L1 = G.N1 + 2 * E1;
    if (t >= d1_points(G)) return;
    const int i = (int)(t % G.N0);
    const long r = t / G.N0;
    const int p0 = i + G.NG, p1 = (int)(r % L1) - E1 + G.NG, p2 = (int)(r / L1) - E2 + G.NG;
    const long idx = p0 + (long)G.n0 * (p1 + (long)G.n1 * p2);
    const bool ycol = AX < 0 && p1 >= G.NG && p1 < G.NG + G.N1;
#pragma unroll
    for (int q = 0; q < N_D1; q++) {
        const double* f = y + (long)d1gf(q) * G.T + idx;
        d1x[(long)q * G.T + idx] = d1r<ORD>(f, 1);
        if (ycol) d1y[(long)q * G.T + idx] = d1r<ORD>(f, G.n0);
    }
}

// one pure-outer ghost point of an RK stage: radiation condition and the stage epilogue
// (SHORT1: as the enclosing kernel's interior points, see ssp_first_short)
template <int FAM, int ORD, bool SHORT1 = false>
__device__ __forceinline__ void outer_point_stage(const GridK& G, const OuterPt p, const double* __restrict__ yin,
                                                  double* out, const double* yn, double* acc,
                                                  const double* __restrict__ finf, const double* __restrict__ wspeed,
                                                  const Stage& st)
{
    const long idx = p.idx;
    const long s2 = (long)G.n0 * G.n1;
    const int k0 = p.kind & 0xff, k2 = (p.kind >> 8) & 0xff;
    double k[NGF];
#pragma unroll
    for (int g = 0; g < NGF; g++) {
        const double* f = yin + (long)g * G.T + idx;
        double rad;
        if constexpr (ORD == 8) {
            rad = p.w0 * osraw8(f, 1, k0);
            if constexpr (FAM == FAM_CYL) rad = fma(p.w2, osraw8(f, s2, k2), rad);
        } else {
            rad = p.w0 * osraw(f, 1, k0);
            if constexpr (FAM == FAM_CYL) rad = fma(p.w2, osraw(f, s2, k2), rad);
        }
        k[g] = -ld(wspeed + g) * fma(ld(f) - ld(finf + g), p.invr, rad);
    }
    stage_store<SHORT1>(st, G.T, idx, k, yin, yn, out, acc);
}

// y[ghost] = p * y[source] for gridfunction g; the sign is applied to the bit pattern (exact)
__device__ __forceinline__ void inner_copy(long T, const InnerPt p, int g, double* y)
{
    const long long sgn = (long long)((p.negmask >> gf_type(g)) & 1) << 63;
    const double v = y[(long)g * T + p.src];
    y[(long)g * T + p.dst] = __longlong_as_double(__double_as_longlong(v) ^ sgn);
}

}  // namespace nrk
