// nr_internal.h -- structures shared by the host side of libnrgpu and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/nr.h"

namespace nrk {

// Per-axis 1D reference-metric arrays (device pointers), one value per
// padded index.  Spherical-like: ax0 = {1/r', 1/r, r''/r'^2, r},
// ax1 = {1/sin th, cot th, sin th, cos th}, ax2 = {sin ph, cos ph}.
// Cylindrical-like: ax0 = {1/rho', 1/rho, rho''/rho'^2, rho},
// ax1 = {sin ph, cos ph}, ax2 = {1/z', z''/z'^2, z}.
struct Rfm {
    const double* ax0;
    const double* ax1;
    const double* ax2;
};

// Launch-invariant description of one grid, passed by value to kernels.
struct GridK {
    int n0, n1, n2;     // padded sizes
    int N0, N1, N2;     // interior sizes
    int NG;
    int fam;            // FAM_SPH / FAM_CYL
    int ax;             // azimuthal axis when it holds two points (1 cylindrical-like, 2 spherical-like), else -1
    int ord;            // finite-difference order N_FD = 2 (NG - 1): 4 or 8
    long T;
    double inv_d1[3];   // 1/(den1 dxx_k): 1/12 (4th order) or 1/840 (8th order) over the spacing
    double inv_d2[3];   // 1/(den2 dxx_k^2): den2 = 12 or 5040
    double sigma_metric;  // Kreiss-Oliger strength on gridfunctions 0-16 (h, a, W, K, lambda)
    double sigma_gauge;   // and on 17-23 (vet, bet, alpha)
    double eta;
    Rfm rfm;
};

// Pure-outer ghost point: radiation condition data (precomputed on the host).
struct OuterPt {
    int idx;            // flat index
    int kind;           // one-sided stencil kind, axis 0 (low byte) and axis 2 (next byte)
    double w0, w2;      // (x^j/r) dxx^d/dx^j / (12 dxx_d) for d = 0, 2
    double invr;        // 1/r
};

// Inner ghost point: parity copy.
struct InnerPt {
    int dst, src;
    int negmask;        // bit t set: parity -1 for tensor type t
    int pad;
};

enum { MODE_RHS = 0, MODE_STAGE1 = 1, MODE_STAGE23 = 2, MODE_STAGE4 = 3, MODE_SSP = 4 };

// Stage description for the fused epilogues.  RK4: stages 1-3 y_next = y_n +
// cnext k and acc (=|+=) cacc k; stage 4 y_n = acc + cacc k.  SSPRK3 (MODE_SSP):
// y_next = cyn y_n + cacc (y_in + cnext k), cnext = dt.
struct Stage {
    int mode;
    int enforce;
    double cnext;
    double cacc;
    double cyn;
    // last stage of nr_step_io: the new state of every computed point also goes to the
    // caller's mapped host buffer, compact layout mirror[g * mirror_n + rank[idx]]
    double* mirror = nullptr;
    const int* rank = nullptr;
    long mirror_n = 0;
};

// Pure-outer points whose radiation condition runs inside the k_rhs launch
// of an RK stage (extra blocks ahead of the interior tiles).
struct OuterArgs {
    const OuterPt* pts = nullptr;
    int npts = 0;
    int nblocks = 0;    // set by launch_rhs
    const double* finf = nullptr;
    const double* wspeed = nullptr;
};

// kernel launchers (nr_kernels.cu)
// k_d1 on yin into d1x / d1y (N_D1 sets of T doubles each; d1y used on general
// grids only), then k_rhs
cudaError_t launch_rhs(const GridK& G, const double* yin, double* d1x, double* d1y, double* out, const double* yn,
                       double* acc, Stage st, cudaStream_t s, OuterArgs oa = OuterArgs());
// k_rhs runs as many blocks as fit on the device at once, each striding over the tiles; this fills
// that count for every k_rhs instantiation on the current device (idempotent, not capture-safe: grid
// creation calls it; until then a launch outside a capture does)
cudaError_t rhs_kernels_init();
cudaError_t launch_outer(const GridK& G, const OuterPt* pts, int npts, const double* yin, double* out,
                         const double* yn, double* acc, const double* finf, const double* wspeed, Stage st,
                         cudaStream_t s);
cudaError_t launch_inner(const GridK& G, const InnerPt* pts, int npts, double* y, cudaStream_t s);
// gather (src: 24-gf set, dst: compact [gf][t]) or scatter (the reverse) over the canonical points
cudaError_t launch_compact(const GridK& G, const int* canon, long nc, const double* src, double* dst, bool gather,
                           cudaStream_t s);
// ctr: perturbation counter per canonical point (NULL: its flat index in G)
cudaError_t launch_bl(const GridK& G, const int* canon_idx, long ncanon, int np, const double* mxyz, double amp,
                      uint64_t seed, double* y, cudaStream_t s, const int* ctr = nullptr);
cudaError_t launch_ham(const GridK& G, const double* y, double* H, double rmin, double rmax, double* partials,
                       int nparts, double* result, cudaStream_t s);
cudaError_t launch_mom(const GridK& G, const double* y, double* M, double rmin, double rmax, double* partials,
                       int nparts, double* result, cudaStream_t s);
int ham_partials_needed(const GridK& G);
cudaError_t launch_finite(const GridK& G, const double* y, int* flag, cudaStream_t s);
// 64-bit digest of the 24 gridfunctions of y at the canonical points canon[0..nc) into *out; ctr: the
// key of each point (NULL: its flat index in G)
cudaError_t launch_digest(const GridK& G, const int* canon, long nc, const double* y, unsigned long long* out,
                          cudaStream_t s, const int* ctr = nullptr);
cudaError_t launch_fp64_probe(int blocks, int iters, double* sink, cudaStream_t s);
cudaError_t launch_ham_reduce(const double* partials, int nparts, double* result, cudaStream_t s);

// records a thread-local error message for nr_last_error() and returns code
int nrk_fail(int code, const char* fmt, ...);

// host-side description of a grid's logical coordinates
struct HostGeom {
    int coords, fam;
    int N[3], n[3], NG;
    long T;
    double dxx[3], lo[3];
    double xx(int d, int i) const { return lo[d] + ((double)(i - NG) + 0.5) * dxx[d]; }
};

// Host-side set-up of one grid, as nr_grid_create computes it before touching the device:
// boundary maps, per-axis reference-metric arrays (layout of Rfm), radiation-condition data of
// the pure-outer points and parity copies of the inner ghosts (flat indices of the padded grid;
// the inner ghosts the RK-stage stencils read first), the canonical points and the CFL step.
// K is complete but for its device pointers (rfm).
struct HostSetup {
    HostGeom G;
    GridK K;
    std::vector<int32_t> src, cls;
    std::vector<int8_t> par;
    std::vector<double> a0, a1, a2;
    std::vector<OuterPt> outer;
    std::vector<InnerPt> inner;
    int n_inner_stencil = 0;
    std::vector<int> canon;
    std::vector<double> cart_canon;
    double dt = 0.0;
};
int host_setup(int coords, const int Nxx[3], const nr_params& P, HostSetup& H);

}  // namespace nrk

// a grid from its host-side set-up H (its vectors are moved from): device buffers allocated and
// uploaded on P.device (nr_grid_create = host_setup + grid_from_setup)
namespace nrk {
int grid_from_setup(HostSetup& H, const nr_params& P, nr_grid** out);
}

// one grid: host maps, device buffers and the CUDA-graph RK4 driver state
struct nr_grid {
    nrk::HostGeom geo;
    nr_params P;
    nrk::GridK K;
    cudaStream_t stream = nullptr;   // user stream (may be the legacy stream)
    cudaStream_t cap = nullptr;      // internal stream used for graph capture
    int device = 0;
    // device buffers
    double *y = nullptr, *ya = nullptr, *yb = nullptr, *acc = nullptr;
    double *ax0 = nullptr, *ax1 = nullptr, *ax2 = nullptr;
    double *d1x = nullptr, *d1y = nullptr;   // stored first differences (k_d1), N_D1 sets each
    nrk::OuterPt* outer = nullptr;
    nrk::InnerPt* inner = nullptr;
    int* canon = nullptr;
    double* finf = nullptr;
    double* wspeed = nullptr;
    double* partials = nullptr;
    double* hres = nullptr;
    int* flag = nullptr;
    unsigned long long* digest = nullptr;
    double* mxyz = nullptr;
    double* stage = nullptr;   // compact-state staging for host transfers (allocated on first use)
    int* crank = nullptr;      // compact position of each point, -1 at inner ghosts (first nr_step_io)
    int n_outer = 0, n_inner = 0, nparts = 0;
    // inner ghosts read by the stencils of an RK stage: the first n_inner_stencil
    // entries of inner (all of them unless the azimuth holds two points; then the
    // azimuthal ghosts, read by nothing within a step, are refreshed on demand)
    int n_inner_stencil = 0;
    // the azimuthal ghosts of the grid-owned state (entries n_inner_stencil.. of inner) lag
    // behind after nr_rk4_step / nr_ssprk3_step; refresh_ghosts copies them before any use
    bool ghosts_stale = false;
    long n_canon = 0;
    size_t bytes = 0;
    double dt_cfl = 0.0;
    // host copies
    std::vector<nrk::InnerPt> inner_h;   // the inner list as uploaded (stencil-read entries first)
    std::vector<int32_t> src, cls;
    std::vector<int8_t> par;
    std::vector<double> cart_canon;  // for the puncture-distance check
    // graph
    cudaGraphExec_t exec = nullptr;
    double graph_dt = 0.0;
    cudaGraphExec_t exec_ssp = nullptr;   // SSPRK3 step
    double graph_dt_ssp = 0.0;
};

// A C-ABI entry point returns a status; no C++ exception (a failed host allocation)
// may cross the C boundary.
template <class F>
int nrk_guard(const char* fn, F&& body) noexcept
{
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return nrk::nrk_fail(NR_ENOMEM, "%s: host memory exhausted", fn);
    } catch (const std::exception& e) {
        return nrk::nrk_fail(NR_EINVAL, "%s: %s", fn, e.what());
    } catch (...) {
        return nrk::nrk_fail(NR_EINVAL, "%s: unexpected error", fn);
    }
}

// the parity copies of the grid-owned state that the integrators leave stale (azimuthal
// ghosts of a two-point azimuth, read by no stencil of a step); stream-ordered
inline cudaError_t refresh_ghosts(nr_grid* g)
{
    if (!g->ghosts_stale) return cudaSuccess;
    g->ghosts_stale = false;
    return nrk::launch_inner(g->K, g->inner + g->n_inner_stencil, g->n_inner - g->n_inner_stencil, g->y, g->stream);
}


