// nr_batch_kernels.cuh -- the per-substage kernel of batched mode and its
// launch helpers, instantiated once per coordinate family (nr_batch_sph.cu,
// nr_batch_cyl.cu) so the two compile in parallel.
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
    int pad;
    Stage st[4];
};

struct BInner {
    int grid, dst, src, negmask;
};

__device__ __forceinline__ void stage_buffers(const BGrid& B, int stage, const double*& yin, double*& out,
                                              const double*& yn)
{
    switch (stage) {
    case 0: yin = B.y; out = B.ya; yn = B.y; break;
    case 1: yin = B.ya; out = B.yb; yn = B.y; break;
    case 2: yin = B.yb; out = B.ya; yn = B.y; break;
    default: yin = B.ya; out = B.y; yn = nullptr; break;
    }
}

template <int FAM, int AX, int TX, int TY>
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
            rhs_point_stage<FAM, AX, true, 4>(B.K, yin, B.d1x, B.d1y, out, yn, B.acc, B.st[stage], i, j);
    } else {
        const int p = (w - B.w_rhs_end) * (TX * TY) + tid;
        if (p < B.n_outer)
            outer_point_stage<FAM, 4>(B.K, B.outer[p], yin, out, yn, B.acc, B.finf, B.wspeed, B.st[stage]);
    }
}

// the stored first differences of every grid's stage input, 256 points per block
template <int AX>
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
    d1_point<AX, 4>(B.K, yin, B.d1x, B.d1y, (long)(w - B.d1_begin) * 256 + threadIdx.x);
}

// tile shapes the autotuner tries (threads per block = TX * TY)
struct TileShape {
    int tx, ty;
};
constexpr TileShape kTiles[] = {{32, 4}, {64, 2}, {128, 1}, {16, 8}, {32, 2}, {64, 1}, {32, 1}};
constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

template <int FAM, int AX, int TX, int TY>
cudaError_t launch_bstage(const BGrid* g, int n, int total, int stage, cudaStream_t s)
{
    if (total > 0) k_batch_stage<FAM, AX, TX, TY><<<total, TX * TY, 0, s>>>(g, n, total, stage);
    return cudaGetLastError();
}

template <int AX>
cudaError_t launch_batch_d1(const BGrid* g, int n, int total_d1, int stage, cudaStream_t s)
{
    if (total_d1 > 0) k_batch_d1<AX><<<total_d1, 256, 0, s>>>(g, n, total_d1, stage);
    return cudaGetLastError();
}

template <int FAM, int AX>
cudaError_t dispatch_stage(int tile, const BGrid* g, int n, int total, int stage, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_bstage<FAM, AX, 32, 4>(g, n, total, stage, s);
    case 1: return launch_bstage<FAM, AX, 64, 2>(g, n, total, stage, s);
    case 2: return launch_bstage<FAM, AX, 128, 1>(g, n, total, stage, s);
    case 3: return launch_bstage<FAM, AX, 16, 8>(g, n, total, stage, s);
    case 4: return launch_bstage<FAM, AX, 32, 2>(g, n, total, stage, s);
    case 5: return launch_bstage<FAM, AX, 64, 1>(g, n, total, stage, s);
    default: return launch_bstage<FAM, AX, 32, 1>(g, n, total, stage, s);
    }
}

// per-family entry points (nr_batch_sph.cu, nr_batch_cyl.cu); two_point: the
// grids' azimuth holds two points (GridK::ax >= 0)
cudaError_t batch_stage_launch_sph(bool two_point, int tile, const BGrid* g, int n, int total, int stage,
                                   cudaStream_t s);
cudaError_t batch_stage_launch_cyl(bool two_point, int tile, const BGrid* g, int n, int total, int stage,
                                   cudaStream_t s);
cudaError_t batch_d1_launch_sph(bool two_point, const BGrid* g, int n, int total_d1, int stage, cudaStream_t s);
cudaError_t batch_d1_launch_cyl(bool two_point, const BGrid* g, int n, int total_d1, int stage, cudaStream_t s);

}  // namespace nrk
