// nr_psi4.cu -- the Weyl scalar psi4 and its spin-weight -2 decomposition on
// spheres (the waveform extraction of Sec. 4.1).
//
// psi4 = -(E_ij - i B_ij) mbar^i mbar^j from the 3+1 electric and magnetic parts
// of the Weyl tensor (vacuum):
//   E_ij = R_ij - K_ik K^k_j + K K_ij,   B_ij = eps_(i|^kl D_k K_l|j),
// with R_ij = Rbar_ij + R^phi_ij (Rbar_ij as in the evolution equations),
// K_ij = W^-2 (Abar_ij + gammabar_ij K/3), D the physical covariant derivative,
// and m = (u_theta + i u_phi)/sqrt 2 from Gram-Schmidt, in the physical metric,
// of the radial, theta and phi directions of the point's Cartesian position.
// Everything is evaluated in the orthonormal reference frame of the rescaled
// variables; the physical connection there is the rotation generators plus
// Delta^m_kl plus the conformal terms 2 (delta^m_k d_l phi + delta^m_l d_k phi -
// gammabar_kl gammabar^mn d_n phi).
//
// Modes C_lm = integral of psi4 conj(-2Y_lm): psi4 is sampled at Gauss-Legendre
// (cos theta) x uniform (phi) nodes of a sphere by cubic Lagrange interpolation
// in the logical coordinates, then each mode is one fixed-order block reduction.
// Node positions, interpolation stencils and w_q -2Y_lm are set up on the host;
// the harmonics come from Wigner's small-d matrix,
// -2Y_lm = sqrt((2l+1)/(4 pi)) d^l_{m,2}(theta) e^{i m phi}.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bssn_point.cuh"
#include "nr_geo.cuh"
#include "nr_internal.h"

namespace nrk {

template <int FAM, int ORD>
__device__ __forceinline__ void psi4_core(const PointIn& P, const double tet[3][3], double& re, double& im)
{
    MetricPart M;
    metric_part<FAM, false, -1, false, ORD>(P, M);
    const double* y = P.y;
    const long T = P.T;
    const Geo& g = P.g;
    const long* st = P.st;
    auto F = [&](int gf) { return y + (long)gf * T; };
    const double* h = M.h;
    const double* gi = M.gi;
    const double W = M.W, iW = M.iW, iW2 = iW * iW;
    double a[6], gf6[6];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        a[s] = ld(F(G_ADD + s));
        gf6[s] = (spi(s) == spj(s) ? 1.0 : 0.0) + h[s];
    }
    const double K = ld(F(G_TRK));
    // K_ij and its frame derivatives e_k K_ij = W^-2 (e_k X + 4 e_k phi X), X = a + gammabar K/3
    double X[6], Kd[6], DK[3][6];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        X[s] = fma(gf6[s], K * (1.0 / 3.0), a[s]);
        Kd[s] = X[s] * iW2;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double eK = g.D[k] * d1r<ORD>(F(G_TRK), st[k]);
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const double eX = fma(M.dh[k][s], K * (1.0 / 3.0), fma(gf6[s], eK * (1.0 / 3.0), g.D[k] * d1r<ORD>(F(G_ADD + s), st[k])));
            DK[k][s] = fma(4.0 * M.dphi[k], X[s], eX) * iW2;
        }
    }
    // Dhat_k K_ij: add the rotation generators
    oms<FAM, 1>(g, 1.0, Kd, DK[1]);
    oms<FAM, 2>(g, 1.0, Kd, DK[2]);
    // physical minus reference connection Q^m_kl
    double gdphi[3];   // gammabar^mn d_n phi
#pragma unroll
    for (int m = 0; m < 3; m++)
        gdphi[m] = fma(gsym(gi, m, 2), M.dphi[2], fma(gsym(gi, m, 1), M.dphi[1], gsym(gi, m, 0) * M.dphi[0]));
    auto Q = [&](int m, int k, int l) {
        double q = M.Dup[m][sp(k, l)] - 2.0 * gsym(gf6, k, l) * gdphi[m];
        if (m == k) q += 2.0 * M.dphi[l];
        if (m == l) q += 2.0 * M.dphi[k];
        return q;
    };
    double DKp[3][6];   // D_k K_ij (physical)
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int s = 0; s < 6; s++) {
            const int i = spi(s), j = spj(s);
            double t = DK[k][s];
#pragma unroll
            for (int m = 0; m < 3; m++) t -= Q(m, k, i) * gsym(Kd, m, j) + Q(m, k, j) * gsym(Kd, i, m);
            DKp[k][s] = t;
        }
    // R_ij = Rbar_ij + R^phi_ij; E_ij
    double lap = 0.0, gp = 0.0;
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const double w = offd(s) ? 2.0 : 1.0;
        lap = fma(w * gi[s], M.DDphir[s], lap);
        gp = fma(w * gi[s], M.dphi[spi(s)] * M.dphi[spj(s)], gp);
    }
    double E[6];
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const int i = spi(s), j = spj(s);
        // with Dbar_i Dbar_j phi = DDphir_ij + 2 e_i phi e_j phi, the e_i phi e_j phi terms cancel
        const double Rphi = -2.0 * M.DDphir[s] - 2.0 * gf6[s] * (lap + 4.0 * gp);
        // K_ik gamma^kl K_lj, gamma^kl = W^2 gammabar^kl
        double kk = 0.0;
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int l = 0; l < 3; l++) kk = fma(gsym(Kd, i, k) * gsym(gi, k, l), gsym(Kd, l, j), kk);
        E[s] = M.Ric[s] + Rphi - W * W * kk + K * Kd[s];
    }
    // B: eps_i^kl D_k K_lj = gamma_im V^m_j / sqrt(det gamma), V^m_j = [mkl] D_k K_lj
    double V[3][3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        V[0][j] = DKp[1][sp(2, j)] - DKp[2][sp(1, j)];
        V[1][j] = DKp[2][sp(0, j)] - DKp[0][sp(2, j)];
        V[2][j] = DKp[0][sp(1, j)] - DKp[1][sp(0, j)];
    }
    const double detb = gf6[0] * (gf6[3] * gf6[5] - gf6[4] * gf6[4]) - gf6[1] * (gf6[1] * gf6[5] - gf6[4] * gf6[2]) +
                        gf6[2] * (gf6[1] * gf6[4] - gf6[3] * gf6[2]);
    const double isq = W * W * W / sqrt(detb);   // 1/sqrt(det gamma), det gamma = det gammabar / W^6
    double Bm[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double t = 0.0;
#pragma unroll
            for (int m = 0; m < 3; m++) t = fma(gsym(gf6, i, m), V[m][j], t);
            Bm[i][j] = t * iW2 * isq;
        }
    // tetrad: Gram-Schmidt of the radial, theta, phi directions in gamma_ij = W^-2 gammabar_ij
    double u[3][3];
    auto dotg = [&](const double* p, const double* q) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) t = fma(gsym(gf6, i, j) * p[i], q[j], t);
        return t * iW2;
    };
#pragma unroll
    for (int A = 0; A < 3; A++) {
#pragma unroll
        for (int d = 0; d < 3; d++) u[A][d] = tet[A][d];
#pragma unroll
        for (int Bq = 0; Bq < A; Bq++) {
            const double c = dotg(u[A], u[Bq]);
#pragma unroll
            for (int d = 0; d < 3; d++) u[A][d] -= c * u[Bq][d];
        }
        const double nrm = 1.0 / sqrt(dotg(u[A], u[A]));
#pragma unroll
        for (int d = 0; d < 3; d++) u[A][d] *= nrm;
    }
    auto proj = [&](const double* p, const double* q, bool isB) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) t = fma(isB ? 0.5 * (Bm[i][j] + Bm[j][i]) : E[sp(i, j)], p[i] * q[j], t);
        return t;
    };
    const double Ett = proj(u[1], u[1], false), Epp = proj(u[2], u[2], false), Etp = proj(u[1], u[2], false);
    const double Btt = proj(u[1], u[1], true), Bpp = proj(u[2], u[2], true), Btp = proj(u[1], u[2], true);
    re = -0.5 * (Ett - Epp) + Btp;
    im = Etp + 0.5 * (Btt - Bpp);
}

constexpr int PSI4_THREADS = 128;

template <int FAM, int ORD>
__global__ void __launch_bounds__(PSI4_THREADS) k_psi4(GridK G, const double* __restrict__ y, double* psi4)
{
    const long t = (long)blockIdx.x * PSI4_THREADS + threadIdx.x;
    if (t >= (long)G.N0 * G.N1 * G.N2) return;
    const int i = (int)(t % G.N0), j = (int)(t / G.N0);
    const int p0 = i + G.NG, p1 = j % G.N1 + G.NG, p2 = j / G.N1 + G.NG;
    const long idx = p0 + (long)G.n0 * (p1 + (long)G.n1 * p2);
    PointIn P;
    P.y = y + idx;
    P.T = G.T;
    P.st[0] = 1;
    P.st[1] = G.n0;
    P.st[2] = (long)G.n0 * G.n1;
    P.ox = 0;
    P.dx = nullptr;
    P.dy = nullptr;
    P.g = make_geo<FAM>(G, p0, p1, p2);
    // the spherical directions of the Cartesian position in the reference frame
    double tet[3][3];
    if constexpr (FAM == FAM_SPH) {
        for (int A = 0; A < 3; A++)
            for (int d = 0; d < 3; d++) tet[A][d] = A == d ? 1.0 : 0.0;
    } else {
        double x[3];
        cart_of(G, p0, p1, p2, x);
        const double rho = sqrt(x[0] * x[0] + x[1] * x[1]), r = sqrt(rho * rho + x[2] * x[2]);
        const double st = rho / r, ct = x[2] / r;
        const double v[3][3] = {{st, 0.0, ct}, {ct, 0.0, -st}, {0.0, 1.0, 0.0}};
        for (int A = 0; A < 3; A++)
            for (int d = 0; d < 3; d++) tet[A][d] = v[A][d];
    }
    double re, im;
    psi4_core<FAM, ORD>(P, tet, re, im);
    psi4[idx] = re;
    psi4[G.T + idx] = im;
}

// psi4 is a scalar: an inner ghost takes the value of the point it maps to
__global__ void __launch_bounds__(256) k_psi4_ghosts(long T, const InnerPt* __restrict__ pts, int npts, double* psi4)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    const InnerPt p = pts[t];
    psi4[p.dst] = psi4[p.src];
    psi4[T + p.dst] = psi4[T + p.src];
}

struct SpherePt {
    long base;         // flat index of the (0,0,0) corner of the 4x4x4 stencil
    double w[3][4];    // cubic Lagrange weights per axis
};

__global__ void __launch_bounds__(128) k_sphere_sample(const double* __restrict__ f, long T, int n0, int n1,
                                                        const SpherePt* __restrict__ pts, int nq, double* samples)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const SpherePt p = pts[q];
    double vr = 0.0, vi = 0.0;
    for (int c = 0; c < 4; c++)
        for (int b = 0; b < 4; b++) {
            const double wbc = p.w[1][b] * p.w[2][c];
            for (int a = 0; a < 4; a++) {
                const long idx = p.base + a + (long)n0 * (b + (long)n1 * c);
                const double w = p.w[0][a] * wbc;
                vr = fma(w, f[idx], vr);
                vi = fma(w, f[T + idx], vi);
            }
        }
    samples[2 * q] = vr;
    samples[2 * q + 1] = vi;
}

// one block per mode: sum_q psi4_q conj(w_q Y_q) in a fixed order
__global__ void __launch_bounds__(256) k_sphere_modes(const double* __restrict__ samples,
                                                       const double* __restrict__ wy, int nq, double* out)
{
    const int mode = blockIdx.x;
    const double* yq = wy + 2L * mode * nq;
    double sr = 0.0, si = 0.0;
    for (int q = threadIdx.x; q < nq; q += 256) {
        const double pr = samples[2 * q], pi = samples[2 * q + 1], yr = yq[2 * q], yi = yq[2 * q + 1];
        sr = fma(pr, yr, fma(pi, yi, sr));
        si = fma(pi, yr, fma(-pr, yi, si));
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = sr;
    sh[1][threadIdx.x] = si;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * mode] = sh[0][0];
        out[2 * mode + 1] = sh[1][0];
    }
}

}  // namespace nrk

using namespace nrk;

namespace {

struct DevGuard {
    int prev = 0;
    explicit DevGuard(int d) { cudaGetDevice(&prev); cudaSetDevice(d); }
    ~DevGuard() { cudaSetDevice(prev); }
};

#define CUDA_TRY(x)                                                                                \
    do {                                                                                           \
        cudaError_t e_ = (x);                                                                      \
        if (e_ != cudaSuccess) return nrk_fail(NR_ECUDA, "%s: %s", #x, cudaGetErrorString(e_));   \
    } while (0)

cudaError_t launch_psi4(const nr_grid* g, const double* y, double* psi4, cudaStream_t s)
{
    const GridK& G = g->K;
    const long n = (long)G.N0 * G.N1 * G.N2;
    const unsigned b = (unsigned)((n + PSI4_THREADS - 1) / PSI4_THREADS);
    if (G.fam == FAM_SPH) {
        if (G.ord == 8) k_psi4<FAM_SPH, 8><<<b, PSI4_THREADS, 0, s>>>(G, y, psi4);
        else k_psi4<FAM_SPH, 4><<<b, PSI4_THREADS, 0, s>>>(G, y, psi4);
    } else {
        if (G.ord == 8) k_psi4<FAM_CYL, 8><<<b, PSI4_THREADS, 0, s>>>(G, y, psi4);
        else k_psi4<FAM_CYL, 4><<<b, PSI4_THREADS, 0, s>>>(G, y, psi4);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || g->n_inner == 0) return e;
    k_psi4_ghosts<<<(g->n_inner + 255) / 256, 256, 0, s>>>(G.T, g->inner, g->n_inner, psi4);
    return cudaGetLastError();
}

// Wigner small-d matrix element d^l_{mp,m}(beta), explicit sum
double wigner_d(int l, int mp, int m, double beta)
{
    auto lf = [](int n) { return lgamma((double)n + 1.0); };
    const double c = cos(0.5 * beta), s = sin(0.5 * beta);
    double sum = 0.0;
    for (int k = std::max(0, m - mp); k <= std::min(l + m, l - mp); k++) {
        const double lg = 0.5 * (lf(l + mp) + lf(l - mp) + lf(l + m) + lf(l - m)) - lf(l + m - k) - lf(k) -
                          lf(l - k - mp) - lf(k - m + mp);
        const int pc = 2 * l - 2 * k + m - mp, ps = 2 * k - m + mp;
        sum += (((k - m + mp) & 1) ? -1.0 : 1.0) * exp(lg) * pow(c, pc) * pow(s, ps);
    }
    return sum;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n
void gl_nodes(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// logical coordinates of a Cartesian point (canonical branch), per coordinate family
void logical_of(const nr_grid* g, const double c[3], double xx[3])
{
    const nr_params& P = g->P;
    auto inv_sinh = [](double A, double w, double v) { return w * asinh(v * sinh(1.0 / w) / A); };
    if (g->geo.fam == FAM_CYL) {
        xx[0] = inv_sinh(P.ampl[0], P.sinhw[0], sqrt(c[0] * c[0] + c[1] * c[1]));
        xx[1] = atan2(c[1], c[0]);
        xx[2] = inv_sinh(P.ampl[2], P.sinhw[2], c[2]);
    } else {
        const double r = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        xx[0] = g->geo.coords == NR_SPHERICAL ? r / P.ampl[0] : inv_sinh(P.ampl[0], P.sinhw[0], r);
        xx[1] = atan2(sqrt(c[0] * c[0] + c[1] * c[1]), c[2]);
        xx[2] = atan2(c[1], c[0]);
    }
}

}  // namespace

extern "C" {

int nr_psi4(nr_grid* g, const double* y_dev, double* psi4_dev)
{
    if (!g || !psi4_dev) return nrk_fail(NR_EINVAL, "bad nr_psi4 arguments");
    DevGuard dg(g->device);
    if (!y_dev) CUDA_TRY(refresh_ghosts(g));
    CUDA_TRY(cudaMemsetAsync(psi4_dev, 0, sizeof(double) * 2 * g->geo.T, g->stream));
    CUDA_TRY(launch_psi4(g, y_dev ? y_dev : g->y, psi4_dev, g->stream));
    return NR_OK;
}

static int nr_psi4_modes_body(nr_grid* g, const double* y_dev, double Rext, int ntheta, int nphi, int lmax, double* modes_out)
{
    if (!g || !modes_out || !(Rext > 0.0) || ntheta < 1 || nphi < 1 || lmax < 2 || lmax > 16 ||
        (long)ntheta * nphi > (1L << 24))
        return nrk_fail(NR_EINVAL, "bad nr_psi4_modes arguments");
    const HostGeom& G = g->geo;
    // sphere nodes, their interpolation stencils and w_q -2Y_lm(theta_q, phi_q)
    std::vector<double> x, w;
    gl_nodes(ntheta, x, w);
    const int nq = ntheta * nphi;
    int nmodes = 0;
    for (int l = 2; l <= lmax; l++) nmodes += 2 * l + 1;
    if ((long)nmodes * nq > (1L << 26))
        return nrk_fail(NR_EINVAL, "nr_psi4_modes: %d modes x %d nodes exceed the 2^26 harmonic table entries", nmodes,
                        nq);
    std::vector<SpherePt> pts(nq);
    std::vector<double> wy(2L * nmodes * nq);
    // w_q sqrt((2l+1)/4pi) d^l_{m,2}(theta) depends on the theta node only
    std::vector<double> amp((size_t)ntheta * nmodes);
    for (int it = 0; it < ntheta; it++) {
        const double th = acos(x[it]), dw = w[it] * 2.0 * M_PI / nphi;
        int md = 0;
        for (int l = 2; l <= lmax; l++)
            for (int m = -l; m <= l; m++, md++)
                amp[(size_t)it * nmodes + md] = sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) * wigner_d(l, m, 2, th) * dw;
    }
    for (int it = 0; it < ntheta; it++)
        for (int jp = 0; jp < nphi; jp++) {
            const int q = it * nphi + jp;
            const double th = acos(x[it]), ph = -M_PI + 2.0 * M_PI * (jp + 0.5) / nphi;
            const double c[3] = {Rext * sin(th) * cos(ph), Rext * sin(th) * sin(ph), Rext * cos(th)};
            double xx[3];
            logical_of(g, c, xx);
            long base = 0, stride = 1;
            for (int d = 0; d < 3; d++) {
                const double fi = (xx[d] - G.lo[d]) / G.dxx[d] + G.NG - 0.5;
                const int i0 = (int)floor(fi);
                const double t = fi - i0;
                if (i0 - 1 < 0 || i0 + 2 >= G.n[d])
                    return nrk_fail(NR_EINVAL, "sphere of radius %g leaves the grid along axis %d", Rext, d);
                // the radial (and, cylindrical, the z) stencil stays on interior points
                const bool outer_axis = d == 0 || (G.fam == FAM_CYL && d == 2);
                if (outer_axis && i0 + 2 > G.NG + G.N[d] - 1)
                    return nrk_fail(NR_EINVAL, "sphere of radius %g reaches the outer boundary", Rext);
                if (G.fam == FAM_CYL && d == 2 && i0 - 1 < G.NG)
                    return nrk_fail(NR_EINVAL, "sphere of radius %g reaches the outer boundary", Rext);
                pts[q].w[d][0] = -t * (t - 1.0) * (t - 2.0) / 6.0;
                pts[q].w[d][1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
                pts[q].w[d][2] = -(t + 1.0) * t * (t - 2.0) / 2.0;
                pts[q].w[d][3] = (t + 1.0) * t * (t - 1.0) / 6.0;
                base += (long)(i0 - 1) * stride;
                stride *= G.n[d];
            }
            pts[q].base = base;
            int md = 0;
            for (int l = 2; l <= lmax; l++)
                for (int m = -l; m <= l; m++, md++) {
                    const double a = amp[(size_t)it * nmodes + md];
                    wy[2L * (md * (long)nq + q)] = a * cos(m * ph);
                    wy[2L * (md * (long)nq + q) + 1] = a * sin(m * ph);
                }
        }
    DevGuard dg(g->device);
    if (!y_dev) CUDA_TRY(refresh_ghosts(g));
    double *psi4 = nullptr, *samples = nullptr, *dwy = nullptr, *dout = nullptr;
    SpherePt* dpts = nullptr;
    cudaError_t e = cudaMalloc(&psi4, sizeof(double) * 2 * G.T);
    if (e == cudaSuccess) e = cudaMalloc(&samples, sizeof(double) * 2 * nq);
    if (e == cudaSuccess) e = cudaMalloc(&dwy, sizeof(double) * wy.size());
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * 2 * nmodes);
    if (e == cudaSuccess) e = cudaMalloc(&dpts, sizeof(SpherePt) * nq);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dwy, wy.data(), sizeof(double) * wy.size(), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dpts, pts.data(), sizeof(SpherePt) * nq, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(psi4, 0, sizeof(double) * 2 * G.T, g->stream);
    if (e == cudaSuccess) e = launch_psi4(g, y_dev ? y_dev : g->y, psi4, g->stream);
    if (e == cudaSuccess) {
        k_sphere_sample<<<(nq + 127) / 128, 128, 0, g->stream>>>(psi4, G.T, G.n[0], G.n[1], dpts, nq, samples);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_sphere_modes<<<nmodes, 256, 0, g->stream>>>(samples, dwy, nq, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(modes_out, dout, sizeof(double) * 2 * nmodes, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    cudaFree(psi4);
    cudaFree(samples);
    cudaFree(dwy);
    cudaFree(dout);
    cudaFree(dpts);
    if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "nr_psi4_modes: %s", cudaGetErrorString(e));
    return NR_OK;
}

int nr_psi4_modes(nr_grid* g, const double* y_dev, double Rext, int ntheta, int nphi, int lmax, double* modes_out)
{
    return nrk_guard("nr_psi4_modes",
                     [&] { return nr_psi4_modes_body(g, y_dev, Rext, ntheta, nphi, lmax, modes_out); });
}

}  // extern "C"
