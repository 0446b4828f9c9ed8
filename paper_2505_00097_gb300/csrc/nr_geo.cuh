// nr_geo.cuh -- per-point geometry from the per-axis reference-metric arrays:
// the frame factors of bssn_point.cuh (make_geo) and Cartesian positions (cart_of).
#pragma once

#include "bssn_point.cuh"
#include "nr_internal.h"

namespace nrk {

template <int FAM>
__device__ __forceinline__ Geo make_geo(const GridK& G, int i0, int i1, int i2)
{
    Geo g;
    const double* A0 = G.rfm.ax0;
    const double s0 = ld(A0 + i0), a = ld(A0 + G.n0 + i0);
    g.d00 = ld(A0 + 2 * G.n0 + i0);
    g.a = a;
    double s2;
    if constexpr (FAM == FAM_SPH) {
        const double isn = ld(G.rfm.ax1 + i1), cot = ld(G.rfm.ax1 + G.n1 + i1);
        s2 = a * isn;
        g.b = a;
        g.c = a * cot;
        g.d22 = 0.0;
        g.e0a = -a * a;
        g.e0b = g.e0a;
        g.e0c = -a * g.c;
        g.e1c = -s2 * s2;
    } else {
        s2 = ld(G.rfm.ax2 + i2);
        g.d22 = ld(G.rfm.ax2 + G.n2 + i2);
        g.b = 0.0;
        g.c = 0.0;
        g.e0a = -a * a;
        g.e0b = 0.0;
        g.e0c = 0.0;
        g.e1c = 0.0;
    }
    g.D[0] = s0 * G.inv_d1[0];
    g.D[1] = a * G.inv_d1[1];
    g.D[2] = s2 * G.inv_d1[2];
    g.D2[0] = s0 * s0 * G.inv_d2[0];
    g.D2[1] = a * a * G.inv_d2[1];
    g.D2[2] = s2 * s2 * G.inv_d2[2];
    g.DD[0] = g.D[0] * g.D[1];
    g.DD[1] = g.D[0] * g.D[2];
    g.DD[2] = g.D[1] * g.D[2];
    return g;
}

__device__ __forceinline__ void cart_of(const GridK& G, int i0, int i1, int i2, double x[3])
{
    if (G.fam == FAM_SPH) {
        const double r = G.rfm.ax0[3 * G.n0 + i0];
        const double st = G.rfm.ax1[2 * G.n1 + i1], ct = G.rfm.ax1[3 * G.n1 + i1];
        const double sp_ = G.rfm.ax2[i2], cp = G.rfm.ax2[G.n2 + i2];
        x[0] = r * st * cp;
        x[1] = r * st * sp_;
        x[2] = r * ct;
    } else {
        const double rho = G.rfm.ax0[3 * G.n0 + i0];
        const double sp_ = G.rfm.ax1[i1], cp = G.rfm.ax1[G.n1 + i1];
        x[0] = rho * cp;
        x[1] = rho * sp_;
        x[2] = G.rfm.ax2[2 * G.n2 + i2];
    }
}

}  // namespace nrk
