// nr_batch_kernels.cuh -- the persistent per-substage kernel of batched mode
// and its launch helpers, instantiated once per coordinate family
// (nr_batch_sph.cu, nr_batch_cyl.cu) so the two compile in parallel.
//
// A work item is either a TX x TY tile of one grid's interior points or a
// chunk of TX*TY of its pure-outer ghost points.  Blocks of the persistent
// kernel take items from an atomic counter until the list is exhausted (a
// bounded loop: each block stops at the first index past the end).  Every
// point runs the same per-point code as the single-grid kernels
// (nr_stage.cuh, with the same two-point-azimuth specialisation AX; the grids
// of one batch share it), so a grid's state after n batched steps is bitwise
// the state after n single-grid steps, whatever the tile shape or the company.
#pragma once

#include <algorithm>

#include "nr_stage.cuh"

namespace nrk {

struct BGrid {
    GridK K;
    double *y, *ya, *yb, *acc;
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
                                                         int* counter, int stage)
{
    __shared__ int s_w;
    const int tid = threadIdx.x;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_w = atomicAdd(counter, 1);
        __syncthreads();
        const int w = s_w;
        if (w >= total) return;
        int lo = 0, hi = ngrids - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (grids[mid].w_begin <= w) lo = mid;
            else hi = mid - 1;
        }
        const BGrid& B = grids[lo];
        const double* yin;
        const double* yn;
        double* out;
        stage_buffers(B, stage, yin, out, yn);
        if (w < B.w_rhs_end) {
            const int t = w - B.w_begin;
            const int i = (t % B.tiles_x) * TX + tid % TX;
            const int j = (t / B.tiles_x) * TY + tid / TX;
            if (i < B.K.N0 && j < B.K.N1 * B.K.N2) rhs_point_stage<FAM, AX>(B.K, yin, out, yn, B.acc, B.st[stage], i, j);
        } else {
            const int p = (w - B.w_rhs_end) * (TX * TY) + tid;
            if (p < B.n_outer)
                outer_point_stage<FAM>(B.K, B.outer[p], yin, out, yn, B.acc, B.finf, B.wspeed, B.st[stage]);
        }
    }
}

// tile shapes the autotuner tries (threads per block = TX * TY)
struct TileShape {
    int tx, ty;
};
constexpr TileShape kTiles[] = {{32, 4}, {64, 2}, {128, 1}, {16, 8}, {32, 2}, {64, 1}, {32, 1}};
constexpr int kNumTiles = sizeof(kTiles) / sizeof(kTiles[0]);

template <int FAM, int AX, int TX, int TY>
cudaError_t launch_bstage(const BGrid* g, int n, int total, int* counter, int stage, int blocks, cudaStream_t s)
{
    k_batch_stage<FAM, AX, TX, TY><<<blocks, TX * TY, 0, s>>>(g, n, total, counter, stage);
    return cudaGetLastError();
}

template <int FAM, int AX, int TX, int TY>
int occupancy_blocks(int sms)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_stage<FAM, AX, TX, TY>, TX * TY, 0) != cudaSuccess)
        return 0;
    return std::max(nb, 1) * sms;
}

template <int FAM, int AX>
cudaError_t dispatch_stage(int tile, const BGrid* g, int n, int total, int* counter, int stage, int blocks,
                           cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_bstage<FAM, AX, 32, 4>(g, n, total, counter, stage, blocks, s);
    case 1: return launch_bstage<FAM, AX, 64, 2>(g, n, total, counter, stage, blocks, s);
    case 2: return launch_bstage<FAM, AX, 128, 1>(g, n, total, counter, stage, blocks, s);
    case 3: return launch_bstage<FAM, AX, 16, 8>(g, n, total, counter, stage, blocks, s);
    case 4: return launch_bstage<FAM, AX, 32, 2>(g, n, total, counter, stage, blocks, s);
    case 5: return launch_bstage<FAM, AX, 64, 1>(g, n, total, counter, stage, blocks, s);
    default: return launch_bstage<FAM, AX, 32, 1>(g, n, total, counter, stage, blocks, s);
    }
}

template <int FAM, int AX>
int dispatch_occupancy(int tile, int sms)
{
    switch (tile) {
    case 0: return occupancy_blocks<FAM, AX, 32, 4>(sms);
    case 1: return occupancy_blocks<FAM, AX, 64, 2>(sms);
    case 2: return occupancy_blocks<FAM, AX, 128, 1>(sms);
    case 3: return occupancy_blocks<FAM, AX, 16, 8>(sms);
    case 4: return occupancy_blocks<FAM, AX, 32, 2>(sms);
    case 5: return occupancy_blocks<FAM, AX, 64, 1>(sms);
    default: return occupancy_blocks<FAM, AX, 32, 1>(sms);
    }
}

// per-family entry points (nr_batch_sph.cu, nr_batch_cyl.cu); two_point: the
// grids' azimuth holds two points (GridK::ax >= 0)
cudaError_t batch_stage_launch_sph(bool two_point, int tile, const BGrid* g, int n, int total, int* counter, int stage,
                                   int blocks, cudaStream_t s);
cudaError_t batch_stage_launch_cyl(bool two_point, int tile, const BGrid* g, int n, int total, int* counter, int stage,
                                   int blocks, cudaStream_t s);
int batch_occupancy_sph(bool two_point, int tile, int sms);
int batch_occupancy_cyl(bool two_point, int tile, int sms);

}  // namespace nrk
