// nr_kernels.cu -- sm_103a FP64 kernels of the BSSN hot path.
//
//   k_d1      raw first differences along axes 0 (and 1) of the gridfunctions
//             with second derivatives, read by k_rhs for its mixed derivatives
//   k_rhs     interior right-hand side (Sec. 2.1 equations, upwinded advection,
//             Kreiss-Oliger dissipation) with the RK4 stage update and the
//             det(gammabar) enforcement fused into its epilogue; in an RK
//             stage its first blocks also run the radiation condition at the
//             pure-outer ghosts (Sec. 3) with the same epilogue
//   k_outer   the radiation condition alone (nr_apply_bcs)
//   k_inner   parity copies at inner ghosts (Sec. 3), one warp-coalesced gather
//             per gridfunction
//   k_bl      Brill-Lindquist data + SplitMix64 perturbation
//   k_ham     Hamiltonian constraint (Eq. Hconstraint) + per-block norm partials
//   k_mom     momentum constraint (Eq. Mconstraint) + per-block norm partials
//   k_ham_reduce  fixed-order reduction of the partials (both constraints)
//   k_finite  NaN/Inf guard on alpha and W
//   k_digest  64-bit digest of a state at the canonical points (bitwise comparisons)
#include <math.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "bssn_point.cuh"
#include "nr_geo.cuh"
#include "nr_internal.h"
#include "nr_stage.cuh"

namespace nrk {

constexpr int RHS_BX = 32, RHS_BY = 4;

// Raw first differences along axis 0 (and, on a general grid, axis 1) of the N_D1
// gridfunctions with second derivatives, at interior i0 and every row a mixed
// stencil of an interior point reads: i1 and i2 within two points of the interior,
// except along a two-point azimuth (no mixed derivatives there); the axis-1 set at
// interior i1 only.
template <int AX, int ORD>
__global__ void __launch_bounds__(256) k_d1(GridK G, const double* __restrict__ y, double* d1x, double* d1y)
{
    d1_point<AX, ORD>(G, y, d1x, d1y, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// one tile of k_rhs: tile tb < oa.nblocks takes pure-outer points, 128 each; the others tile
// (i0, j = i1 + N1 i2) in 32 x 4 points
template <int FAM, int AX, int ORD>
__device__ __forceinline__ void rhs_tile(const GridK& G, const double* __restrict__ yin, const double* __restrict__ d1x,
                                         const double* __restrict__ d1y, double* out, const double* yn, double* acc,
                                         const Stage& st, const OuterArgs& oa, int tb, int nbx)
{
    if (tb < oa.nblocks) {
        const int t = tb * (RHS_BX * RHS_BY) + threadIdx.y * RHS_BX + threadIdx.x;
        if (t < oa.npts)
            outer_point_stage<FAM, ORD, ssp_first_short<AX>()>(G, oa.pts[t], yin, out, yn, acc, oa.finf, oa.wspeed, st);
        return;
    }
    const int b = tb - oa.nblocks;
    const int i = (b % nbx) * RHS_BX + threadIdx.x;
    const int j = (b / nbx) * RHS_BY + threadIdx.y;
    if (i < G.N0 && j < G.N1 * G.N2) rhs_point_stage<FAM, AX, true, ORD>(G, yin, d1x, d1y, out, yn, acc, st, i, j);
}

// Whether k_rhs runs a grid of the resident blocks, each striding over the tiles (every warp then
// keeps its slot for the whole launch): measured faster for the two-point-azimuth kernels; the
// general kernels, whose loop adds register spills, run one block per tile
template <int AX>
__host__ __device__ constexpr bool rhs_strided()
{
    return AX >= 0;
}

template <int FAM, int AX, int ORD>
__global__ void __launch_bounds__(RHS_BX* RHS_BY) k_rhs(GridK G, const double* __restrict__ yin,
                                                        const double* __restrict__ d1x, const double* __restrict__ d1y,
                                                        double* out, const double* yn, double* acc, Stage st,
                                                        OuterArgs oa)
{
    const int nbx = (G.N0 + RHS_BX - 1) / RHS_BX;
    if constexpr (rhs_strided<AX>()) {
        const int ntiles = oa.nblocks + nbx * ((G.N1 * G.N2 + RHS_BY - 1) / RHS_BY);
#pragma unroll 1
        for (int tb = (int)blockIdx.x; tb < ntiles; tb += (int)gridDim.x)
            rhs_tile<FAM, AX, ORD>(G, yin, d1x, d1y, out, yn, acc, st, oa, tb, nbx);
    } else {
        rhs_tile<FAM, AX, ORD>(G, yin, d1x, d1y, out, yn, acc, st, oa, (int)blockIdx.x, nbx);
    }
}

// k_rhs blocks resident on the whole device, per instantiation (family x azimuth axis x order), by
// device; 0: not yet known (a launch then runs one block per tile).  Filled by rhs_kernels_init.
constexpr int RHS_MAX_DEV = 64;
constexpr int RHS_VARIANTS = 8;
std::atomic<int> g_rhs_resident[RHS_MAX_DEV][RHS_VARIANTS];
std::mutex g_rhs_mu;

template <int FAM, int AX, int ORD>
constexpr int rhs_variant()
{
    return (FAM == FAM_SPH ? 0 : 4) + (AX < 0 ? 0 : 2) + (ORD == 8 ? 1 : 0);
}

template <int FAM, int AX, int ORD>
cudaError_t rhs_init_one(int dev, int nsm)
{
    int occ = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rhs<FAM, AX, ORD>, RHS_BX * RHS_BY, 0);
    if (e != cudaSuccess) return e;
    g_rhs_resident[dev][rhs_variant<FAM, AX, ORD>()].store(occ * nsm);
    return cudaSuccess;
}

template <int FAM, int AX, int ORD>
int rhs_resident()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= RHS_MAX_DEV) return 0;
    return g_rhs_resident[dev][rhs_variant<FAM, AX, ORD>()].load();
}

template <int FAM, int AX, int ORD>
cudaError_t launch_k_rhs(long nb, cudaStream_t s, const GridK& G, const double* yin, double* d1x, double* d1y,
                         double* out, const double* yn, double* acc, const Stage& st, const OuterArgs& oa)
{
    int res = rhs_resident<FAM, AX, ORD>();
    if (res == 0) {
        // first launch on this device outside a stream capture: fill the table now
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            const cudaError_t e = rhs_kernels_init();
            if (e != cudaSuccess) return e;
            res = rhs_resident<FAM, AX, ORD>();
        }
    }
    const dim3 grd((unsigned)(rhs_strided<AX>() && res > 0 && res < nb ? res : nb));
    k_rhs<FAM, AX, ORD><<<grd, dim3(RHS_BX, RHS_BY), 0, s>>>(G, yin, d1x, d1y, out, yn, acc, st, oa);
    return cudaGetLastError();
}

template <int FAM, int ORD>
__global__ void __launch_bounds__(128) k_outer(GridK G, const OuterPt* __restrict__ pts, int npts,
                                               const double* __restrict__ yin, double* out, const double* yn,
                                               double* acc, const double* __restrict__ finf,
                                               const double* __restrict__ wspeed, Stage st)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    outer_point_stage<FAM, ORD>(G, pts[t], yin, out, yn, acc, finf, wspeed, st);
}

__global__ void __launch_bounds__(256) k_inner(long T, const InnerPt* __restrict__ pts, int npts, double* y)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    inner_copy(T, pts[t], blockIdx.y, y);
}

// SplitMix64 (Steele, Lea & Flood 2014) first output for state x
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// ctr (NULL: the flat index itself): the perturbation counter of each canonical point -- its flat
// index on the whole grid when G describes one partition of it
__global__ void k_bl(GridK G, const int* __restrict__ canon, const int* __restrict__ ctr, long ncanon, int np,
                     const double* __restrict__ mxyz, double amp, uint64_t seed, double* y)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncanon) return;
    const long idx = canon[t];
    const uint64_t key = ctr ? (uint64_t)ctr[t] : (uint64_t)idx;
    const int i0 = (int)(idx % G.n0), i1 = (int)((idx / G.n0) % G.n1), i2 = (int)(idx / ((long)G.n0 * G.n1));
    double x[3];
    cart_of(G, i0, i1, i2, x);
    double psi = 1.0;
    for (int q = 0; q < np; q++) {
        const double dx = x[0] - mxyz[4 * q + 1], dy = x[1] - mxyz[4 * q + 2], dz = x[2] - mxyz[4 * q + 3];
        psi += mxyz[4 * q] / (2.0 * sqrt(dx * dx + dy * dy + dz * dz));
    }
    const double w = 1.0 / (psi * psi);
    for (int g = 0; g < NGF; g++) y[(long)g * G.T + idx] = 0.0;
    y[(long)G_CF * G.T + idx] = w;
    y[(long)G_ALPHA * G.T + idx] = w;
    if (amp != 0.0) {
        for (int s = 0; s < 6; s++) {
            const uint64_t u = splitmix64(seed ^ (((uint64_t)(G_HDD + s) << 40) | key));
            y[(long)(G_HDD + s) * G.T + idx] = amp * (2.0 * ((double)(u >> 11) * 0x1.0p-53) - 1.0);
        }
    }
}

constexpr int HAM_THREADS = 128;

// per-block partial norms (sum of squares, max, count) of a constraint, in a fixed order
__device__ __forceinline__ void block_partials(double s2, double mx, double cnt, double* partials)
{
    __shared__ double sh[3][HAM_THREADS];
    sh[0][threadIdx.x] = s2;
    sh[1][threadIdx.x] = mx;
    sh[2][threadIdx.x] = cnt;
    __syncthreads();
    for (int w = HAM_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = sh[0][0];
        partials[3 * blockIdx.x + 1] = sh[1][0];
        partials[3 * blockIdx.x + 2] = sh[2][0];
    }
}

template <int FAM, int ORD>
__global__ void __launch_bounds__(HAM_THREADS) k_ham(GridK G, const double* __restrict__ y, double* H, double rmin,
                                                      double rmax, double* partials)
{
    const long t = (long)blockIdx.x * HAM_THREADS + threadIdx.x;
    const long nint = (long)G.N0 * G.N1 * G.N2;
    double s2 = 0.0, mx = 0.0, cnt = 0.0;
    if (t < nint) {
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
        const double h = ham_core<FAM, ORD>(P);
        if (H) H[idx] = h;
        double x[3];
        cart_of(G, p0, p1, p2, x);
        const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (r >= rmin && r <= rmax) {
            s2 = h * h;
            mx = fabs(h);
            cnt = 1.0;
        }
    }
    block_partials(s2, mx, cnt, partials);
}

// momentum constraint (Eq. Mconstraint): rescaled M^i at interior points (M: 3 gridfunctions, or
// NULL) and per-block partial norms of |M|
template <int FAM, int ORD>
__global__ void __launch_bounds__(HAM_THREADS) k_mom(GridK G, const double* __restrict__ y, double* Mout, double rmin,
                                                      double rmax, double* partials)
{
    const long t = (long)blockIdx.x * HAM_THREADS + threadIdx.x;
    const long nint = (long)G.N0 * G.N1 * G.N2;
    double s2 = 0.0, mx = 0.0, cnt = 0.0;
    if (t < nint) {
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
        double Mv[3];
        const double m = mom_core<FAM, ORD>(P, Mv);
        if (Mout) {
            Mout[idx] = Mv[0];
            Mout[G.T + idx] = Mv[1];
            Mout[2 * G.T + idx] = Mv[2];
        }
        double x[3];
        cart_of(G, p0, p1, p2, x);
        const double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (r >= rmin && r <= rmax) {
            s2 = m * m;
            mx = m;
            cnt = 1.0;
        }
    }
    block_partials(s2, mx, cnt, partials);
}

// one block; fixed order: thread t sums partials t, t+256, ..., then a tree
__global__ void __launch_bounds__(256) k_ham_reduce(const double* __restrict__ partials, int nparts, double* result)
{
    __shared__ double sh[3][256];
    double s = 0.0, m = 0.0, c = 0.0;
    for (int p = threadIdx.x; p < nparts; p += 256) {
        s += partials[3 * p];
        m = fmax(m, partials[3 * p + 1]);
        c += partials[3 * p + 2];
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = m;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + w]);
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double cnt = sh[2][0];
        result[0] = cnt > 0.0 ? sqrt(sh[0][0] / cnt) : 0.0;
        result[1] = sh[1][0];
        result[2] = cnt;
    }
}

__global__ void k_finite(long T, const double* __restrict__ y, int* flag)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const double w = y[(long)G_CF * T + t], a = y[(long)G_ALPHA * T + t];
    if (!isfinite(w) || !isfinite(a)) atomicOr(flag, 1);
}

// Digest of a 24-gridfunction set at the canonical points: the wrapping sum over (gf, point)
// of splitmix64(bits ^ splitmix64((gf << 40) | idx)).  A sum modulo 2^64 does not depend on
// the order of its terms, so the digest does not depend on the launch shape; each term is a
// bijective mix of its value's bits, so a change of one value always changes the digest.
// ctr (NULL: the flat index itself): the key of each canonical point -- its flat index on the
// whole grid when the set is one partition of it.
__global__ void __launch_bounds__(256) k_digest(long T, const int* __restrict__ canon, const int* __restrict__ ctr,
                                                long nc, const double* __restrict__ y, unsigned long long* out)
{
    const int g = blockIdx.y;
    unsigned long long acc = 0;
    for (long t = (long)blockIdx.x * 256 + threadIdx.x; t < nc; t += (long)gridDim.x * 256) {
        const long idx = canon[t];
        const uint64_t key = ctr ? (uint64_t)ctr[t] : (uint64_t)idx;
        const uint64_t v = (uint64_t)__double_as_longlong(y[(long)g * T + idx]);
        acc += splitmix64(v ^ splitmix64(((uint64_t)g << 40) | key));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// FP64 FMA throughput probe: 8 independent FMA chains per thread, a fixed
// number of iterations (no data-dependent trip count), one store per thread.
__global__ void __launch_bounds__(256) k_fp64_probe(int iters, double seed, double* sink)
{
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; q++) a[q] = seed + (double)(threadIdx.x + q);
    const double m = 0.999999999, c = 1e-9;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int q = 0; q < 8; q++) a[q] = fma(a[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; q++) s += a[q];
    sink[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fp64_probe(int blocks, int iters, double* sink, cudaStream_t s)
{
    k_fp64_probe<<<blocks, 256, 0, s>>>(iters, 1.0, sink);
    return cudaGetLastError();
}

// ------------------------------------------------------------ launchers

template <int ORD>
cudaError_t launch_rhs_ord(const GridK& G, const double* yin, double* d1x, double* d1y, double* out,
                           const double* yn, double* acc, Stage st, cudaStream_t s, OuterArgs oa)
{
    // the stored first differences of yin
    {
        const unsigned b = (unsigned)((d1_points(G) + 255) / 256);
        if (G.ax == 1) k_d1<1, ORD><<<b, 256, 0, s>>>(G, yin, d1x, d1y);
        else if (G.ax == 2) k_d1<2, ORD><<<b, 256, 0, s>>>(G, yin, d1x, d1y);
        else k_d1<-1, ORD><<<b, 256, 0, s>>>(G, yin, d1x, d1y);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    oa.nblocks = (oa.npts + RHS_BX * RHS_BY - 1) / (RHS_BX * RHS_BY);
    const long nb = (long)((G.N0 + RHS_BX - 1) / RHS_BX) * ((G.N1 * G.N2 + RHS_BY - 1) / RHS_BY) + oa.nblocks;
    if (G.fam == FAM_SPH) {
        if (G.ax == 2) return launch_k_rhs<FAM_SPH, 2, ORD>(nb, s, G, yin, d1x, d1y, out, yn, acc, st, oa);
        return launch_k_rhs<FAM_SPH, -1, ORD>(nb, s, G, yin, d1x, d1y, out, yn, acc, st, oa);
    }
    if (G.ax == 1) return launch_k_rhs<FAM_CYL, 1, ORD>(nb, s, G, yin, d1x, d1y, out, yn, acc, st, oa);
    return launch_k_rhs<FAM_CYL, -1, ORD>(nb, s, G, yin, d1x, d1y, out, yn, acc, st, oa);
}

// the resident-block table of every k_rhs instantiation on the current device (idempotent; not
// during a stream capture)
cudaError_t rhs_kernels_init()
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= RHS_MAX_DEV) return cudaSuccess;   // launches there run one block per tile
    std::lock_guard<std::mutex> lk(g_rhs_mu);
    bool known = true;
    for (int v = 0; v < RHS_VARIANTS; v++) known = known && g_rhs_resident[dev][v].load() > 0;
    if (known) return cudaSuccess;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = rhs_init_one<FAM_SPH, 2, 4>(dev, nsm)) != cudaSuccess) return e;
    if ((e = rhs_init_one<FAM_SPH, -1, 4>(dev, nsm)) != cudaSuccess) return e;
    if ((e = rhs_init_one<FAM_CYL, 1, 4>(dev, nsm)) != cudaSuccess) return e;
    if ((e = rhs_init_one<FAM_CYL, -1, 4>(dev, nsm)) != cudaSuccess) return e;
    if ((e = rhs_init_one<FAM_SPH, 2, 8>(dev, nsm)) != cudaSuccess) return e;
    if ((e = rhs_init_one<FAM_SPH, -1, 8>(dev, nsm)) != cudaSuccess) return e;
    if ((e = rhs_init_one<FAM_CYL, 1, 8>(dev, nsm)) != cudaSuccess) return e;
    return rhs_init_one<FAM_CYL, -1, 8>(dev, nsm);
}

cudaError_t launch_rhs(const GridK& G, const double* yin, double* d1x, double* d1y, double* out, const double* yn,
                       double* acc, Stage st, cudaStream_t s, OuterArgs oa)
{
    return G.ord == 8 ? launch_rhs_ord<8>(G, yin, d1x, d1y, out, yn, acc, st, s, oa)
                      : launch_rhs_ord<4>(G, yin, d1x, d1y, out, yn, acc, st, s, oa);
}

cudaError_t launch_outer(const GridK& G, const OuterPt* pts, int npts, const double* yin, double* out,
                         const double* yn, double* acc, const double* finf, const double* wspeed, Stage st,
                         cudaStream_t s)
{
    if (npts == 0) return cudaSuccess;
    const int b = 128, n = (npts + b - 1) / b;
    if (G.fam == FAM_SPH) {
        if (G.ord == 8) k_outer<FAM_SPH, 8><<<n, b, 0, s>>>(G, pts, npts, yin, out, yn, acc, finf, wspeed, st);
        else k_outer<FAM_SPH, 4><<<n, b, 0, s>>>(G, pts, npts, yin, out, yn, acc, finf, wspeed, st);
    } else {
        if (G.ord == 8) k_outer<FAM_CYL, 8><<<n, b, 0, s>>>(G, pts, npts, yin, out, yn, acc, finf, wspeed, st);
        else k_outer<FAM_CYL, 4><<<n, b, 0, s>>>(G, pts, npts, yin, out, yn, acc, finf, wspeed, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_inner(const GridK& G, const InnerPt* pts, int npts, double* y, cudaStream_t s)
{
    if (npts == 0) return cudaSuccess;
    dim3 grd((npts + 255) / 256, NGF);
    k_inner<<<grd, 256, 0, s>>>(G.T, pts, npts, y);
    return cudaGetLastError();
}

// compact state: the 24 gridfunctions at the canonical points (interior and pure outer),
// layout [gf][t]; one grid row per gridfunction
__global__ void __launch_bounds__(256) k_gather(long T, const int* __restrict__ canon, long nc,
                                                const double* __restrict__ y, double* __restrict__ out)
{
    const double* src = y + (long)blockIdx.y * T;
    double* dst = out + (long)blockIdx.y * nc;
    for (long t = (long)blockIdx.x * 256 + threadIdx.x; t < nc; t += (long)gridDim.x * 256) dst[t] = src[canon[t]];
}

__global__ void __launch_bounds__(256) k_scatter(long T, const int* __restrict__ canon, long nc,
                                                 const double* __restrict__ in, double* __restrict__ y)
{
    const double* src = in + (long)blockIdx.y * nc;
    double* dst = y + (long)blockIdx.y * T;
    for (long t = (long)blockIdx.x * 256 + threadIdx.x; t < nc; t += (long)gridDim.x * 256) dst[canon[t]] = src[t];
}

cudaError_t launch_compact(const GridK& G, const int* canon, long nc, const double* src, double* dst, bool gather,
                           cudaStream_t s)
{
    if (nc == 0) return cudaSuccess;
    const long bx = std::min<long>((nc + 255) / 256, 4L * 152);
    const dim3 grd((unsigned)bx, NGF);
    if (gather) k_gather<<<grd, 256, 0, s>>>(G.T, canon, nc, src, dst);
    else k_scatter<<<grd, 256, 0, s>>>(G.T, canon, nc, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_bl(const GridK& G, const int* canon_idx, long ncanon, int np, const double* mxyz, double amp,
                      uint64_t seed, double* y, cudaStream_t s, const int* ctr)
{
    const int b = 256;
    const long n = (ncanon + b - 1) / b;
    if (n == 0) return cudaSuccess;
    k_bl<<<(unsigned)n, b, 0, s>>>(G, canon_idx, ctr, ncanon, np, mxyz, amp, seed, y);
    return cudaGetLastError();
}

int ham_partials_needed(const GridK& G)
{
    const long nint = (long)G.N0 * G.N1 * G.N2;
    return (int)((nint + HAM_THREADS - 1) / HAM_THREADS);
}

cudaError_t launch_ham(const GridK& G, const double* y, double* H, double rmin, double rmax, double* partials,
                       int nparts, double* result, cudaStream_t s)
{
    if (G.fam == FAM_SPH) {
        if (G.ord == 8) k_ham<FAM_SPH, 8><<<nparts, HAM_THREADS, 0, s>>>(G, y, H, rmin, rmax, partials);
        else k_ham<FAM_SPH, 4><<<nparts, HAM_THREADS, 0, s>>>(G, y, H, rmin, rmax, partials);
    } else {
        if (G.ord == 8) k_ham<FAM_CYL, 8><<<nparts, HAM_THREADS, 0, s>>>(G, y, H, rmin, rmax, partials);
        else k_ham<FAM_CYL, 4><<<nparts, HAM_THREADS, 0, s>>>(G, y, H, rmin, rmax, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ham_reduce<<<1, 256, 0, s>>>(partials, nparts, result);
    return cudaGetLastError();
}

cudaError_t launch_mom(const GridK& G, const double* y, double* M, double rmin, double rmax, double* partials,
                       int nparts, double* result, cudaStream_t s)
{
    if (G.fam == FAM_SPH) {
        if (G.ord == 8) k_mom<FAM_SPH, 8><<<nparts, HAM_THREADS, 0, s>>>(G, y, M, rmin, rmax, partials);
        else k_mom<FAM_SPH, 4><<<nparts, HAM_THREADS, 0, s>>>(G, y, M, rmin, rmax, partials);
    } else {
        if (G.ord == 8) k_mom<FAM_CYL, 8><<<nparts, HAM_THREADS, 0, s>>>(G, y, M, rmin, rmax, partials);
        else k_mom<FAM_CYL, 4><<<nparts, HAM_THREADS, 0, s>>>(G, y, M, rmin, rmax, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ham_reduce<<<1, 256, 0, s>>>(partials, nparts, result);
    return cudaGetLastError();
}

cudaError_t launch_ham_reduce(const double* partials, int nparts, double* result, cudaStream_t s)
{
    k_ham_reduce<<<1, 256, 0, s>>>(partials, nparts, result);
    return cudaGetLastError();
}

cudaError_t launch_digest(const GridK& G, const int* canon, long nc, const double* y, unsigned long long* out,
                          cudaStream_t s, const int* ctr)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || nc == 0) return e;
    const long bx = std::min<long>((nc + 255) / 256, 2L * 152);
    k_digest<<<dim3((unsigned)bx, NGF), 256, 0, s>>>(G.T, canon, ctr, nc, y, out);
    return cudaGetLastError();
}

cudaError_t launch_finite(const GridK& G, const double* y, int* flag, cudaStream_t s)
{
    const int b = 256;
    k_finite<<<(unsigned)((G.T + b - 1) / b), b, 0, s>>>(G.T, y, flag);
    return cudaGetLastError();
}

}  // namespace nrk
