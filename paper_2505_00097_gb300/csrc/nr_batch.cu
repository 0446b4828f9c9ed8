// nr_batch.cu -- batched mode: many grids of uneven sizes advanced together,
// one launch per RK4 or SSPRK3 substage over the work items of all grids plus
// one parity-copy launch, the whole step captured in a CUDA graph; the tile
// shape is chosen by timing.
//
// The per-substage kernel and its work items: nr_batch_kernels.cuh.
#include <string.h>

#include <algorithm>
#include <vector>

#include "nr_batch_kernels.cuh"

namespace nrk {

__global__ void __launch_bounds__(256) k_batch_inner(const BGrid* __restrict__ grids, const BInner* __restrict__ pts,
                                                      int npts, int stage)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    const BInner q = pts[t];
    const BGrid& B = grids[q.grid];
    const double* yin;
    const double* yn;
    double* out;
    stage_buffers(B, stage, yin, out, yn);
    InnerPt p{q.dst, q.src, q.negmask, 0};
    inner_copy(B.K.T, p, blockIdx.y, out);
}

}  // namespace nrk

using namespace nrk;

struct nr_batch {
    std::vector<nr_grid*> grids;
    int fam = FAM_SPH;
    int ord = 4;              // finite-difference order of all grids
    bool two_point = false;   // the grids' azimuth holds two points
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int tile = 3;             // kTiles index: 16x8, the shape the autotuner picks on the workloads
    int total = 0;
    int total_d1 = 0;          // items of the first-difference pass
    BGrid* d_grids = nullptr;
    BInner* d_inner = nullptr;
    int n_inner_stencil = 0;   // parity copies per stage: the ghosts the stencils read
    std::vector<double> dts;   // dts of the current table
    bool table_ok = false;
    bool table_ssp = false;    // the current table (and graph) is for SSPRK3
    cudaGraphExec_t exec = nullptr;
};

namespace {

struct DevGuard {
    int prev = 0;
    explicit DevGuard(int d) { cudaGetDevice(&prev); cudaSetDevice(d); }
    ~DevGuard() { cudaSetDevice(prev); }
};

// work list and per-grid stage constants for tile shape b->tile, step sizes dts and the
// integrator (ssp: SSPRK3, else RK4)
int build_table(nr_batch* b, const double* dts, bool ssp)
{
    const TileShape ts = kTiles[b->tile];
    std::vector<BGrid> h(b->grids.size());
    int w = 0;
    for (size_t q = 0; q < b->grids.size(); q++) {
        nr_grid* g = b->grids[q];
        BGrid& B = h[q];   // value-initialised by the vector
        B.K = g->K;
        B.y = g->y;
        B.ya = g->ya;
        B.yb = g->yb;
        B.acc = g->acc;
        B.d1x = g->d1x;
        B.d1y = g->d1y;
        B.outer = g->outer;
        B.finf = g->finf;
        B.wspeed = g->wspeed;
        B.n_outer = g->n_outer;
        B.tiles_x = (g->K.N0 + ts.tx - 1) / ts.tx;
        const int tiles_y = (g->K.N1 * g->K.N2 + ts.ty - 1) / ts.ty;
        B.w_begin = w;
        B.w_rhs_end = w + B.tiles_x * tiles_y;
        B.w_end = B.w_rhs_end + (g->n_outer + ts.tx * ts.ty - 1) / (ts.tx * ts.ty);
        w = B.w_end;
        // the same stage constants as the single-grid drivers
        const double dt = dts[q];
        const int enf = g->P.enforce_detgb;
        B.ssp = ssp ? 1 : 0;
        if (ssp) {
            B.st[0] = Stage{MODE_SSP, enf, dt, 1.0, 0.0};
            B.st[1] = Stage{MODE_SSP, enf, dt, 0.25, 0.75};
            B.st[2] = Stage{MODE_SSP, enf, dt, 2.0 / 3.0, 1.0 / 3.0};
        } else {
            B.st[0] = Stage{MODE_STAGE1, enf, 0.5 * dt, dt / 6.0, 0.0};
            B.st[1] = Stage{MODE_STAGE23, enf, 0.5 * dt, dt / 3.0, 0.0};
            B.st[2] = Stage{MODE_STAGE23, enf, dt, dt / 3.0, 0.0};
            B.st[3] = Stage{MODE_STAGE4, enf, 0.0, dt / 6.0, 0.0};
        }
    }
    b->total = w;
    int w1 = 0;
    for (size_t q = 0; q < b->grids.size(); q++) {
        h[q].d1_begin = w1;
        w1 += (int)((d1_points(h[q].K) + 255) / 256);
        h[q].d1_end = w1;
    }
    b->total_d1 = w1;
    cudaError_t e = cudaMemcpy(b->d_grids, h.data(), sizeof(BGrid) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "batch table upload: %s", cudaGetErrorString(e));
    b->dts.assign(dts, dts + b->grids.size());
    b->table_ok = true;
    b->table_ssp = ssp;
    return NR_OK;
}

cudaError_t enqueue_stage_launch(nr_batch* b, int stage, cudaStream_t s)
{
    const int n = (int)b->grids.size();
    const bool tp = b->two_point;
    cudaError_t e;
    if (b->fam == FAM_SPH)
        e = b->ord == 8 ? batch_d1_sph8(tp, b->d_grids, n, b->total_d1, stage, s)
                        : batch_d1_sph4(tp, b->d_grids, n, b->total_d1, stage, s);
    else
        e = b->ord == 8 ? batch_d1_cyl8(tp, b->d_grids, n, b->total_d1, stage, s)
                        : batch_d1_cyl4(tp, b->d_grids, n, b->total_d1, stage, s);
    if (e != cudaSuccess) return e;
    if (b->fam == FAM_SPH)
        return b->ord == 8 ? batch_stage_sph8(tp, b->tile, b->d_grids, n, b->total, stage, s)
                           : batch_stage_sph4(tp, b->tile, b->d_grids, n, b->total, stage, s);
    return b->ord == 8 ? batch_stage_cyl8(tp, b->tile, b->d_grids, n, b->total, stage, s)
                       : batch_stage_cyl4(tp, b->tile, b->d_grids, n, b->total, stage, s);
}

// one step of the table's integrator; every stage copies the ghosts the stencils read (the
// grids' remaining azimuthal copies are refreshed on demand, as after single-grid steps)
cudaError_t enqueue_step(nr_batch* b, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const int nst = b->table_ssp ? 3 : 4;
    for (int stage = 0; stage < nst && e == cudaSuccess; stage++) {
        e = enqueue_stage_launch(b, stage, s);
        const int ninner = b->n_inner_stencil;
        if (e == cudaSuccess && ninner) {
            dim3 grd((ninner + 255) / 256, NR_NGF);
            k_batch_inner<<<grd, 256, 0, s>>>(b->d_grids, b->d_inner, ninner, stage);
            e = cudaGetLastError();
        }
    }
    return e;
}

void drop_graph(nr_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

bool same_dts(const nr_batch* b, const double* dts)
{
    for (size_t q = 0; q < b->grids.size(); q++)
        if (b->dts[q] != dts[q]) return false;
    return true;
}

int batch_steps(nr_batch* b, const double* dts, int nsteps, bool ssp, const char* name)
{
    if (!b || !dts || nsteps < 0) return nrk_fail(NR_EINVAL, "bad %s arguments", name);
    for (size_t q = 0; q < b->grids.size(); q++)
        if (!(dts[q] > 0.0)) return nrk_fail(NR_EINVAL, "dt of grid %zu must be positive", q);
    if (nsteps == 0) return NR_OK;
    DevGuard dg(b->device);
    int rc;
    if (!b->table_ok || b->table_ssp != ssp || !same_dts(b, dts)) {
        drop_graph(b);
        if ((rc = build_table(b, dts, ssp))) return rc;
    }
    if (!b->exec) {
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "capture: %s", cudaGetErrorString(e));
        cudaError_t le = enqueue_step(b, b->cap);
        e = cudaStreamEndCapture(b->cap, &graph);
        if (le != cudaSuccess) return nrk_fail(NR_ECUDA, "batch step: %s", cudaGetErrorString(le));
        if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "capture end: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    for (int n = 0; n < nsteps; n++) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    }
    // the azimuthal ghost copies of two-point grids now lag (refreshed on demand)
    for (nr_grid* g : b->grids) g->ghosts_stale = g->n_inner > g->n_inner_stencil;
    return NR_OK;
}


}  // namespace

extern "C" {

static int nr_batch_create_body(nr_grid* const* grids, int ngrids, nr_batch** out)
{
    if (!out) return nrk_fail(NR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grids || ngrids < 1) return nrk_fail(NR_EINVAL, "no grids");
    for (int q = 0; q < ngrids; q++) {
        if (!grids[q]) return nrk_fail(NR_EINVAL, "grid %d is NULL", q);
        if (grids[q]->device != grids[0]->device) return nrk_fail(NR_EINVAL, "grids on different devices");
        if (grids[q]->K.ord != grids[0]->K.ord)
            return nrk_fail(NR_EINVAL, "grids of the 4th- and the 8th-order scheme cannot share a batch");
        if (grids[q]->stream != grids[0]->stream) return nrk_fail(NR_EINVAL, "the grids of a batch share one stream");
        if (grids[q]->geo.fam != grids[0]->geo.fam)
            return nrk_fail(NR_EINVAL, "grids of spherical-like and cylindrical-like coordinates cannot share a batch");
        if ((grids[q]->K.ax >= 0) != (grids[0]->K.ax >= 0))
            return nrk_fail(NR_EINVAL, "grids whose azimuth holds two points and grids whose azimuth holds more "
                                       "cannot share a batch");
        for (int r = 0; r < q; r++)
            if (grids[r] == grids[q]) return nrk_fail(NR_EINVAL, "grid %d appears twice", q);
    }
    nr_batch* b = new nr_batch();
    try {
        b->grids.assign(grids, grids + ngrids);
        b->fam = grids[0]->geo.fam;
        b->ord = grids[0]->K.ord;
        b->two_point = grids[0]->K.ax >= 0;
        b->device = grids[0]->device;
        b->stream = grids[0]->stream;
        DevGuard dg(b->device);
        // parity copies of all grids that the stage stencils read (every ghost, unless the
        // azimuth holds two points: then its ghosts are refreshed per grid on demand), from
        // each grid's partitioned inner list
        std::vector<BInner> inner;
        for (int q = 0; q < ngrids; q++) {
            const nr_grid* g = grids[q];
            for (int t = 0; t < g->n_inner_stencil; t++) {
                const InnerPt& p = g->inner_h[t];
                inner.push_back(BInner{q, p.dst, p.src, p.negmask});
            }
        }
        b->n_inner_stencil = (int)inner.size();
        cudaError_t e = cudaMalloc(&b->d_grids, sizeof(BGrid) * ngrids);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_inner, sizeof(BInner) * std::max<size_t>(inner.size(), 1));
        if (e == cudaSuccess && !inner.empty())
            e = cudaMemcpy(b->d_inner, inner.data(), sizeof(BInner) * inner.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            nr_batch_destroy(b);
            return nrk_fail(e == cudaErrorMemoryAllocation ? NR_ENOMEM : NR_ECUDA, "batch set-up: %s",
                            cudaGetErrorString(e));
        }
        *out = b;
        return NR_OK;
    } catch (...) {
        nr_batch_destroy(b);
        throw;
    }
}

int nr_batch_create(nr_grid* const* grids, int ngrids, nr_batch** out)
{
    return nrk_guard("nr_batch_create", [&] { return nr_batch_create_body(grids, ngrids, out); });
}

void nr_batch_destroy(nr_batch* b)
{
    if (!b) return;
    DevGuard dg(b->device);
    drop_graph(b);
    if (b->d_grids) cudaFree(b->d_grids);
    if (b->d_inner) cudaFree(b->d_inner);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

int nr_batch_set_tile(nr_batch* b, int tile_x, int tile_y)
{
    if (!b) return nrk_fail(NR_EINVAL, "batch is NULL");
    for (int t = 0; t < kNumTiles; t++)
        if (kTiles[t].tx == tile_x && kTiles[t].ty == tile_y) {
            if (t != b->tile) {
                b->tile = t;
                b->table_ok = false;
                drop_graph(b);
            }
            return NR_OK;
        }
    return nrk_fail(NR_EINVAL, "tile %dx%d is not one of the compiled shapes", tile_x, tile_y);
}

static int nr_batch_autotune_body(nr_batch* b, const double* dts, int* tile_x, int* tile_y, double* best_ms)
{
    if (!b || !dts) return nrk_fail(NR_EINVAL, "bad nr_batch_autotune arguments");
    DevGuard dg(b->device);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1;
    float best_t = 1e30f;
    int rc = NR_OK;
    for (int t = 0; t < kNumTiles && rc == NR_OK; t++) {
        b->tile = t;
        if ((rc = build_table(b, dts, b->table_ssp))) break;
        // stage 1 writes only the stage buffer and the accumulator: the state is untouched
        float tt = 0.f;
        for (int rep = 0; rep < 4; rep++) {
            cudaEventRecord(e0, b->stream);
            cudaError_t e = enqueue_stage_launch(b, 0, b->stream);
            cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = nrk_fail(NR_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tt = rep == 1 ? ms : std::min(tt, ms);
        }
        if (rc == NR_OK && tt < best_t) {
            best_t = tt;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->tile = best;
    drop_graph(b);
    if ((rc = build_table(b, dts, b->table_ssp))) return rc;
    if (tile_x) *tile_x = kTiles[best].tx;
    if (tile_y) *tile_y = kTiles[best].ty;
    if (best_ms) *best_ms = best_t;
    return NR_OK;
}

int nr_batch_autotune(nr_batch* b, const double* dts, int* tile_x, int* tile_y, double* best_ms)
{
    return nrk_guard("nr_batch_autotune", [&] { return nr_batch_autotune_body(b, dts, tile_x, tile_y, best_ms); });
}

static int nr_batch_rk4_step_body(nr_batch* b, const double* dts, int nsteps)
{
    return batch_steps(b, dts, nsteps, false, "nr_batch_rk4_step");
}

int nr_batch_rk4_step(nr_batch* b, const double* dts, int nsteps)
{
    return nrk_guard("nr_batch_rk4_step", [&] { return nr_batch_rk4_step_body(b, dts, nsteps); });
}

static int nr_batch_ssprk3_step_body(nr_batch* b, const double* dts, int nsteps)
{
    return batch_steps(b, dts, nsteps, true, "nr_batch_ssprk3_step");
}

int nr_batch_ssprk3_step(nr_batch* b, const double* dts, int nsteps)
{
    return nrk_guard("nr_batch_ssprk3_step", [&] { return nr_batch_ssprk3_step_body(b, dts, nsteps); });
}

}  // extern "C"
