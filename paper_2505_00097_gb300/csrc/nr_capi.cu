// nr_capi.cu -- host side of libnrgpu: the C ABI of include/nr.h, grid set-up
// (per-axis reference-metric arrays, closed-form boundary maps, CFL step) and
// the CUDA-graph RK4 driver.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "bssn_point.cuh"
#include "nr_internal.h"

using namespace nrk;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_OR_FAIL(call)                                                                         \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(NR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

int fam_of(int coords) { return coords == NR_SINH_CYLINDRICAL ? FAM_CYL : FAM_SPH; }

// ---------------------------------------------------------------- geometry
// Logical domains and the cell-centred grid of Sec. 3; sinh map of Sec. 4.1.

void domain(int coords, double lo[3], double hi[3])
{
    if (coords == NR_SINH_CYLINDRICAL) {
        lo[0] = 0.0; hi[0] = 1.0;
        lo[1] = -M_PI; hi[1] = M_PI;
        lo[2] = -1.0; hi[2] = 1.0;
    } else {
        lo[0] = 0.0; hi[0] = 1.0;
        lo[1] = 0.0; hi[1] = M_PI;
        lo[2] = -M_PI; hi[2] = M_PI;
    }
}

void geom_init(int coords, const int Nxx[3], int NG, HostGeom& G)
{
    double hi[3];
    G.coords = coords;
    G.fam = fam_of(coords);
    G.NG = NG;
    domain(coords, G.lo, hi);
    G.T = 1;
    for (int d = 0; d < 3; d++) {
        G.N[d] = Nxx[d];
        G.n[d] = Nxx[d] + 2 * NG;
        G.dxx[d] = (hi[d] - G.lo[d]) / Nxx[d];
        G.T *= G.n[d];
    }
}

// f(x) = A sinh(x/w)/sinh(1/w) and three derivatives; linear map when sinh_kind == 0
void radial(double A, double w, int sinh_kind, double x, double f[4])
{
    if (sinh_kind) {
        const double s = sinh(1.0 / w), sh = sinh(x / w), ch = cosh(x / w);
        f[0] = A * sh / s;
        f[1] = A * ch / (w * s);
        f[2] = A * sh / (w * w * s);
        f[3] = A * ch / (w * w * w * s);
    } else {
        f[0] = A * x;
        f[1] = A;
        f[2] = 0.0;
        f[3] = 0.0;
    }
}

void axis0_map(const HostGeom& G, const nr_params& p, double x, double f[4])
{
    radial(p.ampl[0], p.sinhw[0], G.coords != NR_SPHERICAL, x, f);
}

// per-axis arrays (layout documented in nr_internal.h)
void build_axes(const HostGeom& G, const nr_params& p, std::vector<double>& a0, std::vector<double>& a1,
                std::vector<double>& a2)
{
    const int n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
    a0.assign(4 * n0, 0.0);
    for (int i = 0; i < n0; i++) {
        double f[4];
        axis0_map(G, p, G.xx(0, i), f);
        a0[i] = 1.0 / f[1];
        a0[n0 + i] = 1.0 / f[0];
        a0[2 * n0 + i] = f[2] / (f[1] * f[1]);
        a0[3 * n0 + i] = f[0];
    }
    if (G.fam == FAM_SPH) {
        a1.assign(4 * n1, 0.0);
        for (int i = 0; i < n1; i++) {
            const double th = G.xx(1, i);
            a1[i] = 1.0 / sin(th);
            a1[n1 + i] = cos(th) / sin(th);
            a1[2 * n1 + i] = sin(th);
            a1[3 * n1 + i] = cos(th);
        }
        a2.assign(2 * n2, 0.0);
        for (int i = 0; i < n2; i++) {
            const double ph = G.xx(2, i);
            a2[i] = sin(ph);
            a2[n2 + i] = cos(ph);
        }
    } else {
        a1.assign(2 * n1, 0.0);
        for (int i = 0; i < n1; i++) {
            const double ph = G.xx(1, i);
            a1[i] = sin(ph);
            a1[n1 + i] = cos(ph);
        }
        a2.assign(3 * n2, 0.0);
        for (int i = 0; i < n2; i++) {
            double f[4];
            radial(p.ampl[2], p.sinhw[2], 1, G.xx(2, i), f);
            a2[i] = 1.0 / f[1];
            a2[n2 + i] = f[2] / (f[1] * f[1]);
            a2[2 * n2 + i] = f[0];
        }
    }
}

// Closed-form boundary maps: mirror the integer indices through r=0 / rho=0
// (with phi -> phi + pi), theta = 0, pi (with phi -> phi + pi) and wrap phi
// periodically; each reflection flips the sign of the rescaled vector
// components it reverses (Sec. 2.2 rescaled basis).
int build_maps_host(const HostGeom& G, std::vector<int32_t>& src, std::vector<int8_t>& par,
                    std::vector<int32_t>& cls)
{
    const int NG = G.NG, n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
    const int Nph = G.fam == FAM_SPH ? G.N[2] : G.N[1];
    src.assign(G.T, 0);
    cls.assign(G.T, 0);
    par.assign(10 * G.T, 1);
    for (int i2 = 0; i2 < n2; i2++)
        for (int i1 = 0; i1 < n1; i1++)
            for (int i0 = 0; i0 < n0; i0++) {
                const long idx = i0 + (long)n0 * (i1 + (long)n1 * i2);
                int j0 = i0, j1 = i1, j2 = i2;
                int p[3] = {1, 1, 1};
                bool half_turn = false;
                if (G.fam == FAM_SPH) {
                    if (j0 < NG) {  // r < 0: (r, th, ph) -> (-r, pi - th, ph + pi)
                        j0 = 2 * NG - 1 - j0;
                        j1 = (G.N[1] + 2 * NG - 1) - j1;
                        j2 += Nph / 2;
                        half_turn = true;
                        p[0] = -p[0];
                        p[2] = -p[2];
                    }
                    // th < 0 or th > pi: reflect, ph + pi; repeated while the ghost layers are
                    // deeper than N_th (each pair of reflections is a shift by 2 N_th, i.e. 2 pi)
                    while (j1 < NG || j1 >= NG + G.N[1]) {
                        j1 = (j1 < NG) ? 2 * NG - 1 - j1 : 2 * (NG + G.N[1]) - 1 - j1;
                        j2 += Nph / 2;
                        half_turn = true;
                        p[1] = -p[1];
                        p[2] = -p[2];
                    }
                    j2 = NG + (((j2 - NG) % G.N[2]) + G.N[2]) % G.N[2];
                } else {
                    if (j0 < NG) {  // rho < 0: (rho, ph, z) -> (-rho, ph + pi, z)
                        j0 = 2 * NG - 1 - j0;
                        j1 += Nph / 2;
                        half_turn = true;
                        p[0] = -p[0];
                        p[1] = -p[1];
                    }
                    j1 = NG + (((j1 - NG) % G.N[1]) + G.N[1]) % G.N[1];
                }
                if (half_turn && (Nph % 2) != 0)
                    return fail(NR_EMAP, "N_phi = %d must be even for the r=0 / axis parity maps", Nph);
                const long sidx = j0 + (long)n0 * (j1 + (long)n1 * j2);
                const bool interior = i0 >= NG && i0 < NG + G.N[0] && i1 >= NG && i1 < NG + G.N[1] && i2 >= NG &&
                                      i2 < NG + G.N[2];
                src[idx] = (int32_t)sidx;
                if (sidx == idx) {
                    cls[idx] = interior ? 0 : 1;
                } else {
                    cls[idx] = 2;
                    int8_t* q = &par[10 * idx];
                    q[0] = 1;
                    q[1] = (int8_t)p[0];
                    q[2] = (int8_t)p[1];
                    q[3] = (int8_t)p[2];
                    q[4] = 1;
                    q[5] = (int8_t)(p[0] * p[1]);
                    q[6] = (int8_t)(p[0] * p[2]);
                    q[7] = 1;
                    q[8] = (int8_t)(p[1] * p[2]);
                    q[9] = 1;
                }
            }
    // sources of inner ghosts are interior or pure-outer points
    for (long idx = 0; idx < G.T; idx++)
        if (cls[idx] == 2 && cls[src[idx]] == 2) return fail(NR_EMAP, "ghost %ld maps onto a ghost", idx);
    return NR_OK;
}

int onesided_kind(int i, int n)
{
    if (i - 2 >= 0 && i + 2 < n) return 0;
    if (i + 2 >= n) return (i + 1 < n && i - 3 >= 0) ? 1 : 2;
    return (i - 1 >= 0) ? 3 : 4;
}

// 8th order: the 9-point window a..a+8 nearest to centred that fits, as w = -a
int onesided_window8(int i, int n)
{
    int a = -4;
    if (a < -i) a = -i;
    if (a > n - 1 - i - 8) a = n - 1 - i - 8;
    return -a;
}

double dt_cfl_host(const HostGeom& G, const nr_params& p)
{
    const int NG = G.NG;
    double m0 = 1e300, m1 = 1e300, m2 = 1e300;
    if (G.fam == FAM_SPH) {
        double rmin = 1e300, smin = 1e300;
        for (int i = NG; i < NG + G.N[0]; i++) {
            double f[4];
            axis0_map(G, p, G.xx(0, i), f);
            m0 = std::min(m0, fabs(f[1]) * G.dxx[0]);
            rmin = std::min(rmin, fabs(f[0]));
        }
        for (int j = NG; j < NG + G.N[1]; j++) smin = std::min(smin, fabs(sin(G.xx(1, j))));
        m1 = rmin * G.dxx[1];
        m2 = rmin * smin * G.dxx[2];
    } else {
        double rmin = 1e300;
        for (int i = NG; i < NG + G.N[0]; i++) {
            double f[4];
            radial(p.ampl[0], p.sinhw[0], 1, G.xx(0, i), f);
            m0 = std::min(m0, fabs(f[1]) * G.dxx[0]);
            rmin = std::min(rmin, fabs(f[0]));
        }
        m1 = rmin * G.dxx[1];
        for (int k = NG; k < NG + G.N[2]; k++) {
            double f[4];
            radial(p.ampl[2], p.sinhw[2], 1, G.xx(2, k), f);
            m2 = std::min(m2, fabs(f[1]) * G.dxx[2]);
        }
    }
    return p.cfl * std::min(m0, std::min(m1, m2));
}

// the azimuthal axis when it holds two points (1 cylindrical-like, 2 spherical-like), else -1
int two_point_axis(const HostGeom& G)
{
    if (G.fam == FAM_CYL && G.N[1] == 2) return 1;
    if (G.fam == FAM_SPH && G.N[2] == 2) return 2;
    return -1;
}

int check_args(int coords, const int Nxx[3], const nr_params* p)
{
    if (coords != NR_SINH_SPHERICAL && coords != NR_SINH_CYLINDRICAL && coords != NR_SPHERICAL)
        return fail(NR_EINVAL, "unknown coordinate system %d", coords);
    if (!Nxx) return fail(NR_EINVAL, "Nxx is NULL");
    if (p && p->NG != 3 && p->NG != 5)
        return fail(NR_EINVAL, "NG must be 3 (4th-order FD) or 5 (8th-order FD), with upwinding; got %d", p->NG);
    if (p && p->integrator != NR_RK4 && p->integrator != NR_SSPRK3)
        return fail(NR_EINVAL, "integrator must be NR_RK4 or NR_SSPRK3; got %d", p->integrator);
    if (p) {
        for (int g = 1; g < NR_NGF; g++) {
            const int first = g < 17 ? 0 : 17;
            if (!(p->ko_sigma[g] == p->ko_sigma[first]))
                return fail(NR_EINVAL, "ko_sigma must take one value on gridfunctions 0-16 (metric) and one on 17-23 "
                                       "(gauge); gridfunction %d differs", g);
        }
        if (!(p->ko_sigma[0] >= 0.0) || !(p->ko_sigma[17] >= 0.0))
            return fail(NR_EINVAL, "ko_sigma must be non-negative");
    }
    const int pad = 2 * (p ? p->NG : 3);
    long T = 1;
    for (int d = 0; d < 3; d++) {
        if (Nxx[d] < 1 || Nxx[d] > (1 << 20)) return fail(NR_EINVAL, "Nxx[%d] = %d out of range", d, Nxx[d]);
        T *= Nxx[d] + pad;
    }
    if (T * 24 >= (1L << 40) || T >= (1L << 31)) return fail(NR_EINVAL, "grid too large (%ld points)", T);
    return NR_OK;
}

}  // namespace

int nrk::nrk_fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// ------------------------------------------------------------------ grid

namespace {

template <typename T>
int dmalloc(nr_grid* g, T** p, size_t count)
{
    const size_t b = sizeof(T) * std::max<size_t>(count, 1);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e != cudaSuccess) return fail(NR_ENOMEM, "cudaMalloc(%zu): %s", b, cudaGetErrorString(e));
    g->bytes += b;
    return NR_OK;
}

void free_grid(nr_grid* g)
{
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->exec_ssp) cudaGraphExecDestroy(g->exec_ssp);
    void* ptrs[] = {g->y, g->ya, g->yb, g->acc, g->d1x, g->d1y, g->ax0, g->ax1, g->ax2, g->outer, g->inner, g->canon,
                    g->finf, g->wspeed, g->partials, g->hres, g->flag, g->digest, g->mxyz, g->stage, g->crank};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (g->cap) cudaStreamDestroy(g->cap);
    cudaSetDevice(prev);
    delete g;
}

struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int dev) { cudaGetDevice(&prev); cudaSetDevice(dev); }
    ~DeviceGuard() { cudaSetDevice(prev); }
};

// one RK stage: interior right-hand side and radiation condition in one launch,
// then the parity copies (ninner: the first entries of the inner list)
int enqueue_stage(nr_grid* g, cudaStream_t s, const double* yin, double* out, const double* yn, double* acc,
                  Stage st, int ninner)
{
    OuterArgs oa;
    oa.pts = g->outer;
    oa.npts = g->n_outer;
    oa.finf = g->finf;
    oa.wspeed = g->wspeed;
    CUDA_OR_FAIL(launch_rhs(g->K, yin, g->d1x, g->d1y, out, yn, acc, st, s, oa));
    CUDA_OR_FAIL(launch_inner(g->K, g->inner, ninner, out, s));
    return NR_OK;
}

// one classic RK4 step: y1 = y + dt/2 k1, y2 = y + dt/2 k2, y3 = y + dt k3,
// y_{n+1} = y + dt/6 (k1 + 2 k2 + 2 k3 + k4), accumulated in acc
// mirror (may be NULL): host-mirror fields for the last stage (nr_step_io)
int enqueue_rk4(nr_grid* g, cudaStream_t s, double dt, const Stage* mirror = nullptr)
{
    const int enf = g->P.enforce_detgb;
    Stage s1{MODE_STAGE1, enf, 0.5 * dt, dt / 6.0, 0.0};
    Stage s2{MODE_STAGE23, enf, 0.5 * dt, dt / 3.0, 0.0};
    Stage s3{MODE_STAGE23, enf, dt, dt / 3.0, 0.0};
    Stage s4{MODE_STAGE4, enf, 0.0, dt / 6.0, 0.0};
    if (mirror) {
        s4.mirror = mirror->mirror;
        s4.rank = mirror->rank;
        s4.mirror_n = mirror->mirror_n;
    }
    int rc;
    // every stage copies only the ghosts the stencils read; the rest of y_{n+1}'s are
    // refreshed on demand (refresh_ghosts)
    const int ns = g->n_inner_stencil;
    if ((rc = enqueue_stage(g, s, g->y, g->ya, g->y, g->acc, s1, ns))) return rc;
    if ((rc = enqueue_stage(g, s, g->ya, g->yb, g->y, g->acc, s2, ns))) return rc;
    if ((rc = enqueue_stage(g, s, g->yb, g->ya, g->y, g->acc, s3, ns))) return rc;
    if ((rc = enqueue_stage(g, s, g->ya, g->y, nullptr, g->acc, s4, ns))) return rc;
    return NR_OK;
}

// one SSPRK3 step (Gottlieb-Shu-Tadmor): y1 = y + dt k(y), y2 = 3/4 y + 1/4 (y1 + dt k(y1)),
// y_{n+1} = 1/3 y + 2/3 (y2 + dt k(y2)), the last stage in place
int enqueue_ssprk3(nr_grid* g, cudaStream_t s, double dt, const Stage* mirror = nullptr)
{
    const int enf = g->P.enforce_detgb;
    Stage s1{MODE_SSP, enf, dt, 1.0, 0.0};
    Stage s2{MODE_SSP, enf, dt, 0.25, 0.75};
    Stage s3{MODE_SSP, enf, dt, 2.0 / 3.0, 1.0 / 3.0};
    if (mirror) {
        s3.mirror = mirror->mirror;
        s3.rank = mirror->rank;
        s3.mirror_n = mirror->mirror_n;
    }
    int rc;
    const int ns = g->n_inner_stencil;
    if ((rc = enqueue_stage(g, s, g->y, g->ya, g->y, nullptr, s1, ns))) return rc;
    if ((rc = enqueue_stage(g, s, g->ya, g->yb, g->y, nullptr, s2, ns))) return rc;
    if ((rc = enqueue_stage(g, s, g->yb, g->y, g->y, nullptr, s3, ns))) return rc;
    return NR_OK;
}

}  // namespace

// Host-side set-up of one grid: everything nr_grid_create computes before it touches the
// device (coordinates, per-axis arrays, boundary maps, radiation-condition data, CFL step).
int nrk::host_setup(int coords, const int Nxx[3], const nr_params& P, HostSetup& H)
{
    int rc = check_args(coords, Nxx, &P);
    if (rc) return rc;
    geom_init(coords, Nxx, P.NG, H.G);
    const HostGeom& G = H.G;
    if ((rc = build_maps_host(G, H.src, H.par, H.cls))) return rc;
    H.dt = dt_cfl_host(G, P);
    std::vector<double>&a0 = H.a0, &a1 = H.a1, &a2 = H.a2;
    build_axes(G, P, a0, a1, a2);
    // radiation-condition data of the pure outer points, parity copies of the inner ghosts
    std::vector<OuterPt>& outer = H.outer;
    std::vector<InnerPt>& inner = H.inner;
    std::vector<int>& canon = H.canon;
    outer.clear();
    inner.clear();
    canon.clear();
    const int n0 = G.n[0], n1 = G.n[1];
    for (long idx = 0; idx < G.T; idx++) {
        const int c = H.cls[idx];
        if (c != 2) canon.push_back((int)idx);
        if (c == 1) {
            const int i0 = (int)(idx % n0), i1 = (int)((idx / n0) % n1), i2 = (int)(idx / ((long)n0 * n1));
            OuterPt o{};
            o.idx = (int)idx;
            double f[4];
            // stencil kind per axis and the denominator of its integer weights
            const bool o8 = G.NG == 5;
            const double den = o8 ? 840.0 : 12.0;
            auto kind = [&](int i, int n) { return o8 ? onesided_window8(i, n) : onesided_kind(i, n); };
            if (G.fam == FAM_SPH) {
                axis0_map(G, P, G.xx(0, i0), f);
                o.kind = kind(i0, G.n[0]);
                o.w0 = (1.0 / f[1]) / (den * G.dxx[0]);
                o.w2 = 0.0;
                o.invr = 1.0 / f[0];
            } else {
                double z[4];
                radial(P.ampl[0], P.sinhw[0], 1, G.xx(0, i0), f);
                radial(P.ampl[2], P.sinhw[2], 1, G.xx(2, i2), z);
                const double r = sqrt(f[0] * f[0] + z[0] * z[0]);
                o.kind = kind(i0, G.n[0]) | (kind(i2, G.n[2]) << 8);
                o.w0 = (f[0] / r) * (1.0 / f[1]) / (den * G.dxx[0]);
                o.w2 = (z[0] / r) * (1.0 / z[1]) / (den * G.dxx[2]);
                o.invr = 1.0 / r;
            }
            (void)i1;
            outer.push_back(o);
        } else if (c == 2) {
            InnerPt q{};
            q.dst = (int)idx;
            q.src = H.src[idx];
            int m = 0;
            for (int t = 0; t < 10; t++)
                if (H.par[10 * idx + t] < 0) m |= 1 << t;
            q.negmask = m;
            inner.push_back(q);
        }
    }
    // ghosts the RK-stage stencils read first: with a two-point azimuth (GridK::ax) the
    // stencils of interior and pure-outer points never reach an azimuthal ghost
    const int ax = two_point_axis(G);
    auto read_by_stencils = [&](const InnerPt& q) {
        if (ax < 0) return true;
        const long idx = q.dst;
        const int ia = ax == 1 ? (int)((idx / n0) % n1) : (int)(idx / ((long)n0 * n1));
        return ia >= G.NG && ia < G.NG + G.N[ax];
    };
    std::stable_partition(inner.begin(), inner.end(), read_by_stencils);
    H.n_inner_stencil = (int)std::count_if(inner.begin(), inner.end(), read_by_stencils);
    // Cartesian positions of canonical points, for the puncture check
    H.cart_canon.resize(3 * canon.size());
    for (size_t t = 0; t < canon.size(); t++) {
        const long idx = canon[t];
        const int i0 = (int)(idx % n0), i1 = (int)((idx / n0) % n1), i2 = (int)(idx / ((long)n0 * n1));
        double* x = &H.cart_canon[3 * t];
        if (G.fam == FAM_SPH) {
            const double r = a0[3 * n0 + i0], st = a1[2 * n1 + i1], ct = a1[3 * n1 + i1];
            const double sp_ = a2[i2], cp = a2[G.n[2] + i2];
            x[0] = r * st * cp;
            x[1] = r * st * sp_;
            x[2] = r * ct;
        } else {
            const double rho = a0[3 * n0 + i0], sp_ = a1[i1], cp = a1[n1 + i1];
            x[0] = rho * cp;
            x[1] = rho * sp_;
            x[2] = a2[2 * G.n[2] + i2];
        }
    }
    GridK& K = H.K;
    memset(&K, 0, sizeof K);
    K.n0 = G.n[0]; K.n1 = G.n[1]; K.n2 = G.n[2];
    K.N0 = G.N[0]; K.N1 = G.N[1]; K.N2 = G.N[2];
    K.NG = G.NG;
    K.fam = G.fam;
    K.ax = two_point_axis(G);
    K.ord = 2 * (G.NG - 1);
    K.T = G.T;
    for (int d = 0; d < 3; d++) {
        // the denominators of the integer stencil weights (bssn_point.cuh, FD<ORD>)
        K.inv_d1[d] = 1.0 / ((K.ord == 8 ? 840.0 : 12.0) * G.dxx[d]);
        K.inv_d2[d] = 1.0 / ((K.ord == 8 ? 5040.0 : 12.0) * G.dxx[d] * G.dxx[d]);
    }
    K.sigma_metric = P.ko_sigma[0];
    K.sigma_gauge = P.ko_sigma[17];
    K.eta = P.eta;
    return NR_OK;
}

extern "C" {

const char* nr_last_error(void) { return g_err.c_str(); }

int nr_params_default(int coords, nr_params* out)
{
    if (!out) return fail(NR_EINVAL, "out is NULL");
    memset(out, 0, sizeof *out);
    const bool cyl = coords == NR_SINH_CYLINDRICAL;
    for (int d = 0; d < 3; d++) {
        out->ampl[d] = cyl ? 300.0 : 10.0;
        out->sinhw[d] = 0.2;
    }
    for (int g = 0; g < NR_NGF; g++) {
        out->ko_sigma[g] = 0.3;
        out->wavespeed[g] = 1.0;
        out->f_inf[g] = (g == G_CF || g == G_ALPHA) ? 1.0 : 0.0;
    }
    out->eta = 2.0;
    out->cfl = 0.5;
    out->h_rmin = 0.0;
    out->h_rmax = 1e300;
    out->NG = 3;
    out->enforce_detgb = 1;
    out->device = 0;
    out->stream = nullptr;
    return NR_OK;
}

static int nr_build_maps_body(int coords, const int Nxx[3], int NG, int32_t* src, int8_t* parity, int32_t* cls)
{
    nr_params p;
    nr_params_default(coords, &p);
    p.NG = NG;
    int rc = check_args(coords, Nxx, &p);
    if (rc) return rc;
    if (!src || !parity || !cls) return fail(NR_EINVAL, "NULL output array");
    HostGeom G;
    geom_init(coords, Nxx, NG, G);
    std::vector<int32_t> s, c;
    std::vector<int8_t> q;
    if ((rc = build_maps_host(G, s, q, c))) return rc;
    memcpy(src, s.data(), sizeof(int32_t) * G.T);
    memcpy(cls, c.data(), sizeof(int32_t) * G.T);
    memcpy(parity, q.data(), 10 * G.T);
    return NR_OK;
}

int nr_build_maps(int coords, const int Nxx[3], int NG, int32_t* src, int8_t* parity, int32_t* cls)
{
    return nrk_guard("nr_build_maps", [&] { return nr_build_maps_body(coords, Nxx, NG, src, parity, cls); });
}

static int nr_dt_cfl_body(int coords, const int Nxx[3], const nr_params* params, double* dt_out)
{
    int rc = check_args(coords, Nxx, params);
    if (rc) return rc;
    if (!params || !dt_out) return fail(NR_EINVAL, "NULL argument");
    HostGeom G;
    geom_init(coords, Nxx, params->NG, G);
    *dt_out = dt_cfl_host(G, *params);
    return NR_OK;
}

int nr_dt_cfl(int coords, const int Nxx[3], const nr_params* params, double* dt_out)
{
    return nrk_guard("nr_dt_cfl", [&] { return nr_dt_cfl_body(coords, Nxx, params, dt_out); });
}

static int nr_grid_create_body(int coords, const int Nxx[3], const nr_params* params, nr_grid** out)
{
    if (!out) return fail(NR_EINVAL, "out is NULL");
    *out = nullptr;
    nr_params P;
    if (params)
        P = *params;
    else
        nr_params_default(coords, &P);
    HostSetup H;
    int rc = host_setup(coords, Nxx, P, H);
    if (rc) return rc;
    return grid_from_setup(H, P, out);
}

}  // extern "C"

// A grid from its host-side set-up (consumed): device buffers allocated and uploaded on P.device.
int nrk::grid_from_setup(HostSetup& H, const nr_params& P, nr_grid** out)
{
    int rc = NR_OK;
    *out = nullptr;
    nr_grid* g = new nr_grid();
    try {
        g->P = P;
        g->device = P.device;
        g->stream = (cudaStream_t)P.stream;
        g->geo = H.G;
        const HostGeom& G = g->geo;
        g->src = std::move(H.src);
        g->par = std::move(H.par);
        g->cls = std::move(H.cls);
        g->dt_cfl = H.dt;
        g->cart_canon = std::move(H.cart_canon);
        g->n_inner_stencil = H.n_inner_stencil;
        g->n_outer = (int)H.outer.size();
        g->n_inner = (int)H.inner.size();
        g->n_canon = (long)H.canon.size();
        const std::vector<double>&a0 = H.a0, &a1 = H.a1, &a2 = H.a2;
        const std::vector<OuterPt>& outer = H.outer;
        const std::vector<InnerPt>& inner = H.inner;
        const std::vector<int>& canon = H.canon;

        DeviceGuard dg(g->device);
        const size_t set = (size_t)NR_NGF * G.T;
        std::vector<double> finf(P.f_inf, P.f_inf + NR_NGF), ws(P.wavespeed, P.wavespeed + NR_NGF);
        GridK& K = g->K;
        K = H.K;
        g->nparts = ham_partials_needed(K);
        if ((rc = dmalloc(g, &g->y, set)) || (rc = dmalloc(g, &g->ya, set)) || (rc = dmalloc(g, &g->yb, set)) ||
            (rc = dmalloc(g, &g->acc, set)) || (rc = dmalloc(g, &g->d1x, (size_t)N_D1 * G.T)) ||
            (rc = dmalloc(g, &g->d1y, K.ax < 0 ? (size_t)N_D1 * G.T : 1)) || (rc = dmalloc(g, &g->ax0, a0.size())) ||
            (rc = dmalloc(g, &g->ax1, a1.size())) || (rc = dmalloc(g, &g->ax2, a2.size())) ||
            (rc = dmalloc(g, &g->outer, outer.size())) || (rc = dmalloc(g, &g->inner, inner.size())) ||
            (rc = dmalloc(g, &g->canon, canon.size())) || (rc = dmalloc(g, &g->finf, NR_NGF)) ||
            (rc = dmalloc(g, &g->wspeed, NR_NGF)) || (rc = dmalloc(g, &g->partials, 3 * (size_t)g->nparts)) ||
            (rc = dmalloc(g, &g->hres, 3)) || (rc = dmalloc(g, &g->flag, 1)) || (rc = dmalloc(g, &g->digest, 1)) ||
            (rc = dmalloc(g, &g->mxyz, 64))) {
            free_grid(g);
            return rc;
        }
        K.rfm.ax0 = g->ax0;
        K.rfm.ax1 = g->ax1;
        K.rfm.ax2 = g->ax2;
        cudaError_t e = cudaSuccess;
        auto up = [&](void* d, const void* h, size_t b) {
            if (e == cudaSuccess && b) e = cudaMemcpy(d, h, b, cudaMemcpyHostToDevice);
        };
        up(g->ax0, a0.data(), sizeof(double) * a0.size());
        up(g->ax1, a1.data(), sizeof(double) * a1.size());
        up(g->ax2, a2.data(), sizeof(double) * a2.size());
        up(g->outer, outer.data(), sizeof(OuterPt) * outer.size());
        up(g->inner, inner.data(), sizeof(InnerPt) * inner.size());
        g->inner_h = inner;
        up(g->canon, canon.data(), sizeof(int) * canon.size());
        up(g->finf, finf.data(), sizeof(double) * NR_NGF);
        up(g->wspeed, ws.data(), sizeof(double) * NR_NGF);
        if (e == cudaSuccess) e = cudaMemset(g->y, 0, sizeof(double) * set);
        if (e == cudaSuccess) e = cudaMemset(g->acc, 0, sizeof(double) * set);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = rhs_kernels_init();   // before any step is captured
        if (e != cudaSuccess) {
            free_grid(g);
            return fail(NR_ECUDA, "grid upload: %s", cudaGetErrorString(e));
        }
        *out = g;
        return NR_OK;
    } catch (...) {
        free_grid(g);
        throw;
    }
}

extern "C" {

int nr_grid_create(int coords, const int Nxx[3], const nr_params* params, nr_grid** out)
{
    return nrk_guard("nr_grid_create", [&] { return nr_grid_create_body(coords, Nxx, params, out); });
}

void nr_grid_destroy(nr_grid* grid) { free_grid(grid); }

int nr_query(const nr_grid* g, nr_grid_info* info)
{
    if (!g || !info) return fail(NR_EINVAL, "NULL argument");
    for (int d = 0; d < 3; d++) {
        info->N[d] = g->geo.N[d];
        info->n[d] = g->geo.n[d];
    }
    info->T = g->geo.T;
    info->interior = (int64_t)g->geo.N[0] * g->geo.N[1] * g->geo.N[2];
    info->n_outer = g->n_outer;
    info->n_inner = g->n_inner;
    info->dt_cfl = g->dt_cfl;
    info->device_bytes = g->bytes;
    info->n_inner_stencil = g->n_inner_stencil;
    // per stage: k_d1, k_rhs (interior + pure-outer points), then k_inner over the ghosts the
    // stencils read, if any (the rest are refreshed on demand, one launch)
    info->launches_per_step = 8 + 4 * (g->n_inner_stencil > 0);
    info->launches_per_ssprk3_step = 6 + 3 * (g->n_inner_stencil > 0);
    info->n_state_points = g->n_canon;
    return NR_OK;
}

static int nr_set_brill_lindquist_body(nr_grid* g, int npunct, const double* mass, const double* xyz, double perturb_amp,
                                       uint64_t seed)
{
    if (!g || npunct < 0 || npunct > 16 || (npunct && (!mass || !xyz)))
        return fail(NR_EINVAL, "bad Brill-Lindquist arguments");
    for (size_t t = 0; t < g->cart_canon.size() / 3; t++)
        for (int q = 0; q < npunct; q++) {
            const double dx = g->cart_canon[3 * t] - xyz[3 * q], dy = g->cart_canon[3 * t + 1] - xyz[3 * q + 1],
                         dz = g->cart_canon[3 * t + 2] - xyz[3 * q + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < 1e-12)
                return fail(NR_EINVAL, "puncture %d lies on a grid point", q);
        }
    DeviceGuard dg(g->device);
    double m[64];
    for (int q = 0; q < npunct; q++) {
        m[4 * q] = mass[q];
        m[4 * q + 1] = xyz[3 * q];
        m[4 * q + 2] = xyz[3 * q + 1];
        m[4 * q + 3] = xyz[3 * q + 2];
    }
    if (npunct) CUDA_OR_FAIL(cudaMemcpyAsync(g->mxyz, m, sizeof(double) * 4 * npunct, cudaMemcpyHostToDevice, g->stream));
    CUDA_OR_FAIL(cudaMemsetAsync(g->y, 0, sizeof(double) * NR_NGF * g->geo.T, g->stream));
    CUDA_OR_FAIL(launch_bl(g->K, g->canon, g->n_canon, npunct, g->mxyz, perturb_amp, seed, g->y, g->stream));
    CUDA_OR_FAIL(launch_inner(g->K, g->inner, g->n_inner, g->y, g->stream));
    g->ghosts_stale = false;
    // the host array m must stay valid until the copy is done
    CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    return NR_OK;
}

int nr_set_brill_lindquist(nr_grid* g, int npunct, const double* mass, const double* xyz, double perturb_amp,
                           uint64_t seed)
{
    return nrk_guard("nr_set_brill_lindquist",
                     [&] { return nr_set_brill_lindquist_body(g, npunct, mass, xyz, perturb_amp, seed); });
}

int nr_rhs(nr_grid* g, const double* y_dev, double* rhs_dev)
{
    if (!g || !y_dev || !rhs_dev || y_dev == rhs_dev) return fail(NR_EINVAL, "bad nr_rhs arguments");
    DeviceGuard dg(g->device);
    Stage st{MODE_RHS, 0, 0.0, 0.0, 0.0};
    CUDA_OR_FAIL(launch_rhs(g->K, y_dev, g->d1x, g->d1y, rhs_dev, nullptr, nullptr, st, g->stream));
    return NR_OK;
}

int nr_apply_bcs(nr_grid* g, const double* y_dev, double* rhs_dev)
{
    if (!g || !y_dev || !rhs_dev || y_dev == rhs_dev) return fail(NR_EINVAL, "bad nr_apply_bcs arguments");
    DeviceGuard dg(g->device);
    Stage st{MODE_RHS, 0, 0.0, 0.0, 0.0};
    CUDA_OR_FAIL(launch_outer(g->K, g->outer, g->n_outer, y_dev, rhs_dev, nullptr, nullptr, g->finf, g->wspeed, st,
                              g->stream));
    CUDA_OR_FAIL(launch_inner(g->K, g->inner, g->n_inner, rhs_dev, g->stream));
    return NR_OK;
}

int nr_apply_inner_bcs(nr_grid* g, double* gfs_dev)
{
    if (!g || !gfs_dev) return fail(NR_EINVAL, "bad nr_apply_inner_bcs arguments");
    DeviceGuard dg(g->device);
    CUDA_OR_FAIL(launch_inner(g->K, g->inner, g->n_inner, gfs_dev, g->stream));
    return NR_OK;
}

int nr_rk4_step(nr_grid* g, double dt, int nsteps)
{
    if (!g || !(dt > 0.0) || nsteps < 0) return fail(NR_EINVAL, "bad nr_rk4_step arguments");
    if (nsteps == 0) return NR_OK;
    DeviceGuard dg(g->device);
    if (!g->exec || g->graph_dt != dt) {
        if (g->exec) {
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
        cudaGraph_t graph;
        CUDA_OR_FAIL(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_rk4(g, g->cap, dt);
        cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(NR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(NR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        g->graph_dt = dt;
    }
    for (int n = 0; n < nsteps; n++) CUDA_OR_FAIL(cudaGraphLaunch(g->exec, g->stream));
    g->ghosts_stale = g->n_inner > g->n_inner_stencil;
    return NR_OK;
}

int nr_ssprk3_step(nr_grid* g, double dt, int nsteps)
{
    if (!g || !(dt > 0.0) || nsteps < 0) return fail(NR_EINVAL, "bad nr_ssprk3_step arguments");
    if (nsteps == 0) return NR_OK;
    DeviceGuard dg(g->device);
    if (!g->exec_ssp || g->graph_dt_ssp != dt) {
        if (g->exec_ssp) {
            cudaGraphExecDestroy(g->exec_ssp);
            g->exec_ssp = nullptr;
        }
        cudaGraph_t graph;
        CUDA_OR_FAIL(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_ssprk3(g, g->cap, dt);
        cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(NR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g->exec_ssp, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(NR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        g->graph_dt_ssp = dt;
    }
    for (int n = 0; n < nsteps; n++) CUDA_OR_FAIL(cudaGraphLaunch(g->exec_ssp, g->stream));
    g->ghosts_stale = g->n_inner > g->n_inner_stencil;
    return NR_OK;
}

int nr_hamiltonian(nr_grid* g, const double* y_dev, double* H_dev, double* l2_out, double* linf_out)
{
    if (!g) return fail(NR_EINVAL, "grid is NULL");
    DeviceGuard dg(g->device);
    if (!y_dev) CUDA_OR_FAIL(refresh_ghosts(g));
    const double* y = y_dev ? y_dev : g->y;
    if (H_dev) CUDA_OR_FAIL(cudaMemsetAsync(H_dev, 0, sizeof(double) * g->geo.T, g->stream));
    CUDA_OR_FAIL(launch_ham(g->K, y, H_dev, g->P.h_rmin, g->P.h_rmax, g->partials, g->nparts, g->hres, g->stream));
    if (l2_out || linf_out) {
        double r[3];
        CUDA_OR_FAIL(cudaMemcpyAsync(r, g->hres, sizeof r, cudaMemcpyDeviceToHost, g->stream));
        CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
        if (l2_out) *l2_out = r[0];
        if (linf_out) *linf_out = r[1];
    }
    return NR_OK;
}

int nr_momentum(nr_grid* g, const double* y_dev, double* M_dev, double* l2_out, double* linf_out)
{
    if (!g) return fail(NR_EINVAL, "grid is NULL");
    DeviceGuard dg(g->device);
    if (!y_dev) CUDA_OR_FAIL(refresh_ghosts(g));
    const double* y = y_dev ? y_dev : g->y;
    if (M_dev) CUDA_OR_FAIL(cudaMemsetAsync(M_dev, 0, sizeof(double) * 3 * g->geo.T, g->stream));
    CUDA_OR_FAIL(launch_mom(g->K, y, M_dev, g->P.h_rmin, g->P.h_rmax, g->partials, g->nparts, g->hres, g->stream));
    if (l2_out || linf_out) {
        double r[3];
        CUDA_OR_FAIL(cudaMemcpyAsync(r, g->hres, sizeof r, cudaMemcpyDeviceToHost, g->stream));
        CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
        if (l2_out) *l2_out = r[0];
        if (linf_out) *linf_out = r[1];
    }
    return NR_OK;
}

int nr_get_state(nr_grid* g, double* dst, int to_host)
{
    if (!g || !dst) return fail(NR_EINVAL, "bad nr_get_state arguments");
    DeviceGuard dg(g->device);
    const size_t b = sizeof(double) * NR_NGF * g->geo.T;
    CUDA_OR_FAIL(refresh_ghosts(g));
    CUDA_OR_FAIL(cudaMemcpyAsync(dst, g->y, b, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream));
    if (to_host) CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    return NR_OK;
}

int nr_set_state(nr_grid* g, const double* src, int from_host)
{
    if (!g || !src) return fail(NR_EINVAL, "bad nr_set_state arguments");
    DeviceGuard dg(g->device);
    const size_t b = sizeof(double) * NR_NGF * g->geo.T;
    g->ghosts_stale = false;
    CUDA_OR_FAIL(cudaMemcpyAsync(g->y, src, b, from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream));
    if (from_host) CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    return NR_OK;
}

int nr_get_state_compact(nr_grid* g, double* dst, int to_host)
{
    if (!g || !dst) return fail(NR_EINVAL, "bad nr_get_state_compact arguments");
    DeviceGuard dg(g->device);
    const long nc = g->n_canon;
    const size_t b = sizeof(double) * NR_NGF * nc;
    if (!to_host) {
        CUDA_OR_FAIL(launch_compact(g->K, g->canon, nc, g->y, dst, true, g->stream));
        return NR_OK;
    }
    if (!g->stage) CUDA_OR_FAIL(cudaMalloc(&g->stage, b));
    CUDA_OR_FAIL(launch_compact(g->K, g->canon, nc, g->y, g->stage, true, g->stream));
    CUDA_OR_FAIL(cudaMemcpyAsync(dst, g->stage, b, cudaMemcpyDeviceToHost, g->stream));
    CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    return NR_OK;
}

// the upload of nr_set_state_compact, enqueued on the grid's stream without waiting for it
static int set_state_compact_async(nr_grid* g, const double* src, int from_host)
{
    const long nc = g->n_canon;
    const size_t b = sizeof(double) * NR_NGF * nc;
    const double* from = src;
    if (from_host) {
        if (!g->stage) CUDA_OR_FAIL(cudaMalloc(&g->stage, b));
        CUDA_OR_FAIL(cudaMemcpyAsync(g->stage, src, b, cudaMemcpyHostToDevice, g->stream));
        from = g->stage;
    }
    CUDA_OR_FAIL(launch_compact(g->K, g->canon, nc, from, g->y, false, g->stream));
    // the ghosts the stencils read now; the azimuthal copies on demand (refresh_ghosts)
    CUDA_OR_FAIL(launch_inner(g->K, g->inner, g->n_inner_stencil, g->y, g->stream));
    g->ghosts_stale = g->n_inner > g->n_inner_stencil;
    return NR_OK;
}

int nr_set_state_compact(nr_grid* g, const double* src, int from_host)
{
    if (!g || !src) return fail(NR_EINVAL, "bad nr_set_state_compact arguments");
    DeviceGuard dg(g->device);
    int rc = set_state_compact_async(g, src, from_host);
    if (rc) return rc;
    if (from_host) CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    return NR_OK;
}

// nr_step_io after the upload: the steps and the read-back
static int step_io_steps(nr_grid* g, int integrator, double dt, int nsteps, double* host_out)
{
    int rc;
    auto steps = [&](int n) { return integrator == NR_SSPRK3 ? nr_ssprk3_step(g, dt, n) : nr_rk4_step(g, dt, n); };
    if (nsteps > 1 && (rc = steps(nsteps - 1))) return rc;
    cudaPointerAttributes a{};
    void* mapped = nullptr;
    if (host_out && cudaPointerGetAttributes(&a, host_out) == cudaSuccess && a.type == cudaMemoryTypeHost)
        mapped = a.devicePointer;
    cudaGetLastError();   // an unregistered pointer leaves no error behind
    if (!mapped) {
        if ((rc = steps(1))) return rc;
        if (host_out) return nr_get_state_compact(g, host_out, 1);
        CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
        return NR_OK;
    }
    if (!g->crank) {
        std::vector<int> r(g->geo.T, -1);
        int t = 0;
        for (long idx = 0; idx < g->geo.T; idx++)
            if (g->cls[idx] != 2) r[idx] = t++;
        CUDA_OR_FAIL(cudaMalloc(&g->crank, sizeof(int) * r.size()));
        CUDA_OR_FAIL(cudaMemcpy(g->crank, r.data(), sizeof(int) * r.size(), cudaMemcpyHostToDevice));
    }
    // the last step launched directly, its last stage writing the compact state to host_out
    Stage m{};
    m.mirror = (double*)mapped;
    m.rank = g->crank;
    m.mirror_n = g->n_canon;
    rc = integrator == NR_SSPRK3 ? enqueue_ssprk3(g, g->stream, dt, &m) : enqueue_rk4(g, g->stream, dt, &m);
    if (rc) return rc;
    g->ghosts_stale = g->n_inner > g->n_inner_stencil;
    CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    return NR_OK;
}

static int nr_step_io_body(nr_grid* g, int integrator, double dt, int nsteps, const double* host_in, double* host_out)
{
    if (!g || !(dt > 0.0) || nsteps < 1 || (integrator != NR_RK4 && integrator != NR_SSPRK3))
        return fail(NR_EINVAL, "bad nr_step_io arguments");
    DeviceGuard dg(g->device);
    // the upload is not waited for: the steps follow it on the same stream, and the call
    // returns only after the stream has drained
    int rc = host_in ? set_state_compact_async(g, host_in, 1) : NR_OK;
    if (rc == NR_OK) rc = step_io_steps(g, integrator, dt, nsteps, host_out);
    // on an error the upload may still be reading host_in: drain the stream before returning
    if (rc != NR_OK && host_in) cudaStreamSynchronize(g->stream);
    return rc;
}

int nr_step_io(nr_grid* g, int integrator, double dt, int nsteps, const double* host_in, double* host_out)
{
    return nrk_guard("nr_step_io", [&] { return nr_step_io_body(g, integrator, dt, nsteps, host_in, host_out); });
}

int nr_sync(nr_grid* g)
{
    if (!g) return fail(NR_EINVAL, "grid is NULL");
    DeviceGuard dg(g->device);
    CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    return NR_OK;
}

int nr_check_finite(nr_grid* g)
{
    if (!g) return fail(NR_EINVAL, "grid is NULL");
    DeviceGuard dg(g->device);
    int h = 0;
    CUDA_OR_FAIL(refresh_ghosts(g));
    CUDA_OR_FAIL(cudaMemsetAsync(g->flag, 0, sizeof(int), g->stream));
    CUDA_OR_FAIL(launch_finite(g->K, g->y, g->flag, g->stream));
    CUDA_OR_FAIL(cudaMemcpyAsync(&h, g->flag, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    if (h) return fail(NR_ENONFINITE, "non-finite alpha or W in the state");
    return NR_OK;
}

int nr_state_digest(nr_grid* g, const double* y_dev, uint64_t* out)
{
    if (!g || !out) return fail(NR_EINVAL, "bad nr_state_digest arguments");
    DeviceGuard dg(g->device);
    unsigned long long h = 0;
    CUDA_OR_FAIL(launch_digest(g->K, g->canon, g->n_canon, y_dev ? y_dev : g->y, g->digest, g->stream));
    CUDA_OR_FAIL(cudaMemcpyAsync(&h, g->digest, sizeof h, cudaMemcpyDeviceToHost, g->stream));
    CUDA_OR_FAIL(cudaStreamSynchronize(g->stream));
    *out = (uint64_t)h;
    return NR_OK;
}

int nr_fp64_peak(int device, double* flops_out)
{
    if (!flops_out) return fail(NR_EINVAL, "flops_out is NULL");
    DeviceGuard dg(device);
    int sms = 0;
    CUDA_OR_FAIL(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int blocks = sms * 8, iters = 4096;
    double* sink = nullptr;
    CUDA_OR_FAIL(cudaMalloc(&sink, sizeof(double) * 256 * (size_t)blocks));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    float best = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 6 && err == cudaSuccess; rep++) {
        cudaEventRecord(e0, s);
        err = launch_fp64_probe(blocks, iters, sink, s);
        cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(sink);
    if (err != cudaSuccess) return fail(NR_ECUDA, "fp64 probe: %s", cudaGetErrorString(err));
    *flops_out = 2.0 * 8.0 * iters * 256.0 * blocks / (best * 1e-3);
    return NR_OK;
}

}  // extern "C"
