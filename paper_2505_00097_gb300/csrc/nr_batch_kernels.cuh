// nr_batch_kernels.cuh -- the per-substage kernel of batched mode and its
// launch helpers, instantiated once per coordinate family and finite-difference
// order (nr_batch_{sph,cyl}{,8}.cu) so the four compile in parallel.
//
// A work item is either a TX x TY tile of one grid's interior points or a
// chunk of TX*TY of its pure-outer ghost points.  One launch per RK substage
// covers the items of all grids, one block per item: the block finds its grid
// by binary search over the items' start indices and stages that grid's
// record in shared memory.  (A persistent variant that took items from an
// atomic counter carried its loop state through the 255-register point code
// and spilled three to four times as much.)  Every
// point runs the same per-point code as the single-grid kernels
// (nr_stage.cuh, with the same two-point-azimuth specialisation AX; the grids
// of one batch share it), so a grid's state after n batched steps is bitwise
// the state after n single-grid steps, whatever the tile shape or the company.
#pragma once

#include <algorithm>

#include "nr_stage.cuh"

namespace nrk {

struct __align__(16) BGrid {
    GridK K;
    double *y, *ya, *yb, *acc;
    double *d1x, *d1y;         // the grid's stored first differences
    int d1_begin, d1_end;      // its items of the first-difference pass (256 points each)
    const OuterPt* outer;
    const double* finf;
    const double* wspeed;
    int n_outer;
    int tiles_x;
    int w_begin, w_rhs_end, w_end;
    int ssp;                   // the table's integrator: 0 RK4 (st[0..3]), 1 SSPRK3 (st[0..2])
    Stage st[4];
};

struct BInner {
    int grid, dst, src, negmask;
};

// the buffers of one substage, as the single-grid drivers use them: RK4 y -> ya -> yb -> ya
// -> y (the last stage from acc); SSPRK3 y -> ya -> yb -> y (in place, reading y_n)
__device__ __forceinline__ void stage_buffers(const BGrid& B, int stage, const double*& yin, double*& out,
                                              const double*& yn)
{
    switch (stage) {
    case 0: yin = B.y; out = B.ya; yn = B.y; break;
    case 1: yin = B.ya; out = B.yb; yn = B.y; break;
    case 2: yin = B.yb; out = B.ssp ? B.y : B.ya; yn = B.y; break;
    default: yin = B.ya; out = B.y; yn = nullptr; break;
    }
}

template <int FAM, int AX, int ORD, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_batch_stage(const BGrid* __restrict__ grids, int ngrids, int total,
                                                         int stage)
{
    // one block per work item; the item's grid record is staged in shared memory
    __shared__ __align__(16) unsigned long long s_grid[(sizeof(BGrid) + 7) / 8];
    const int tid = threadIdx.x;
    const int w = (int)blockIdx.x;
    if (w >= total) return;
    int lo = 0, hi = ngrids - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (grids[mid].w_begin <= w) lo = mid;
        else hi = mid - 1;
    }
    {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(grids + lo);
        for (int q = tid; q < (int)(sizeof(BGrid) / 8); q += TX * TY) s_grid[q] = src[q];
    }
    __syncthreads();
    const BGrid& B = *reinterpret_cast<const BGrid*>(s_grid);
    const double* yin;
    const double* yn;
    double* out;
    stage_buffers(B, stage, yin, out, yn);
    if (w < B.w_rhs_end) {
        const int t = w - B.w_begin;
        const int i = (t % B.tiles_x) * TX + tid % TX;
        const int j = (t / B.tiles_x) * TY + tid / TX;
        if (i < B.K.N0 && j < B.K.N1 * B.K.N2)
            rhs_point_stage<FAM, AX, true, ORD>(B.K, yin, B.d1x, B.d1y, out, yn, B.acc, B.st[stage], i, j);
    } else {
        const int p = (w - B.w_rhs_end) * (TX * TY) + tid;
        if (p < B.n_outer)
            outer_point_stage<FAM, ORD, ssp_first_short<AX>()>(B.K, B.outer[p], yin, out, yn, B.acc, B.finf, B.wspeed,
                                                               B.st[stage]);
    }
}

// the stored first differences of every grid's stage input, 256 points per block
template <int AX, int ORD>
__global__ void __launch_bounds__(256) k_batch_d1(const BGrid* __restrict__ grids, int ngrids, int total, int stage)
{
    const int w = (int)blockIdx.x;
    if (w >= total) return;
    int lo = 0, hi = ngrids - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (grids[mid].d1_begin <= w) lo = mid;
        else hi = mid - 1;
    }
    const BGrid& B = grids[lo];
    const double* yin;
    const double* yn;
    double* out;
    stage_buffers(B, stage, yin, out, yn);
    d1_point<AX, ORD>(B.K, yin, B.d1x, B.d1y, (long)(w - B.d1_begin) * 256 + threadIdx.x);
}

// tile shapes the autotuner tries (threads per block = TX * TY)
struct TileShape {
    int tx, ty;
};
constexpr TileShape kTiles[] = {{32, 4}, {64, 2}, {128, 1}, {16, 8}, {32, 2}, {64, 1}, {32, 1}};
constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

template <int FAM, int AX, int ORD, int TX, int TY>
cudaError_t launch_bstage(const BGrid* g, int n, int total, int stage, cudaStream_t s)
{
    if (total > 0) k_batch_stage<FAM, AX, ORD, TX, TY><<<total, TX * TY, 0, s>>>(g, n, total, stage);
    return cudaGetLastError();
}

template <int AX, int ORD>
cudaError_t launch_batch_d1(const BGrid* g, int n, int total_d1, int stage, cudaStream_t s)
{
    if (total_d1 > 0) k_batch_d1<AX, ORD><<<total_d1, 256, 0, s>>>(g, n, total_d1, stage);
    return cudaGetLastError();
}

template <int FAM, int AX, int ORD>
cudaError_t dispatch_stage(int tile, const BGrid* g, int n, int total, int stage, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_bstage<FAM, AX, ORD, 32, 4>(g, n, total, stage, s);
    case 1: return launch_bstage<FAM, AX, ORD, 64, 2>(g, n, total, stage, s);
    case 2: return launch_bstage<FAM, AX, ORD, 128, 1>(g, n, total, stage, s);
    case 3: return launch_bstage<FAM, AX, ORD, 16, 8>(g, n, total, stage, s);
    case 4: return launch_bstage<FAM, AX, ORD, 32, 2>(g, n, total, stage, s);
    case 5: return launch_bstage<FAM, AX, ORD, 64, 1>(g, n, total, stage, s);
    default: return launch_bstage<FAM, AX, ORD, 32, 1>(g, n, total, stage, s);
    }
}

// one translation unit per family and order (nr_batch_{sph,cyl}{,8}.cu) defines, through
// NRK_BATCH_LAUNCH, the substage launch (tile shape `tile`) and the first-difference pass
// of all grids; two_point: the grids' azimuth holds two points (GridK::ax >= 0)
#define NRK_BATCH_DECL(NAME)                                                                                   \
    cudaError_t batch_stage_##NAME(bool two_point, int tile, const BGrid* g, int n, int total, int stage,      \
                                   cudaStream_t s);                                                            \
    cudaError_t batch_d1_##NAME(bool two_point, const BGrid* g, int n, int total_d1, int stage, cudaStream_t s);
NRK_BATCH_DECL(sph4)
NRK_BATCH_DECL(sph8)
NRK_BATCH_DECL(cyl4)
NRK_BATCH_DECL(cyl8)

#define NRK_BATCH_LAUNCH(NAME, FAM_, AXTWO_, ORD_)                                                             \
    cudaError_t batch_stage_##NAME(bool two_point, int tile, const BGrid* g, int n, int total, int stage,      \
                                   cudaStream_t s)                                                             \
    {                                                                                                          \
        return two_point ? dispatch_stage<FAM_, AXTWO_, ORD_>(tile, g, n, total, stage, s)                     \
                         : dispatch_stage<FAM_, -1, ORD_>(tile, g, n, total, stage, s);                        \
    }                                                                                                          \
    cudaError_t batch_d1_##NAME(bool two_point, const BGrid* g, int n, int total_d1, int stage, cudaStream_t s) \
    {                                                                                                          \
        return two_point ? launch_batch_d1<AXTWO_, ORD_>(g, n, total_d1, stage, s)                             \
                         : launch_batch_d1<-1, ORD_>(g, n, total_d1, stage, s);                                \
    }

}  // namespace nrk
