// nr_server.cu -- served mode: continuous batching of evolution requests.
//
// Requests (one grid + Brill-Lindquist data + a final time each) are queued
// by nr_server_submit.  nr_server_advance makes queued requests resident
// (grid allocated, initial data set) while the summed device bytes stay
// within the HBM budget and a slot is free, then advances a selection of the
// resident requests together, as one nr_batch per kind of grid (coordinate
// family x azimuth kind; one launch per RK4 substage for each).
// The policy orders both steps:
//   FIFO: arrival order;
//   SRPT: least remaining work first (remaining steps x interior points),
//         preemptive at chunk boundaries -- a resident request that is not
//         selected keeps its state in HBM and resumes later.
// The selection is the longest prefix of that order whose interior points sum
// to at most max_batch_points (at least one request; 0 = no cap).  Membership
// changes only at step boundaries: a request that reaches its final time is
// retired (its Hamiltonian-constraint norms recorded, optionally its final
// state copied to the host, its device memory released) and the freed budget
// admits the next queued requests.  Each request advances with its own CFL
// step; since every point runs the single-grid arithmetic, a request's result
// does not depend on which other requests shared the GPU with it, nor on when
// it was paused.
// The host-side set-up of the requests next in line (coordinates, per-axis arrays,
// boundary maps: the part of nr_grid_create that runs on the CPU) is computed
// ahead by a worker thread while the GPU advances the running requests, so
// that admission only allocates, uploads and sets initial data.
// A guard checks alpha and W of the advanced requests for non-finite values
// every few steps (nr_server_set_guard); a request that fails it is retired
// as failed with NR_ENONFINITE while the others keep running.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "nr_internal.h"

using nrk::nrk_fail;

namespace {

struct Request {
    int64_t id = 0;
    int coords = 0;
    int N[3] = {0, 0, 0};
    nr_params P{};
    int np = 0;
    double mass[16] = {0};
    double xyz[48] = {0};
    double t_final = 0.0;
    int keep_state = 0;        // bit 0: keep the final state; bit 1: keep its digest
    size_t bytes = 0;
    int64_t interior = 0;      // interior points
    int64_t steps_est = 0;     // steps to t_final at the CFL step, known at submission
    double submit_t = 0.0;     // submission time (steady clock, seconds)
    // progress
    int status = 0;          // 0 queued, 1 running, 2 done, 3 failed
    nr_grid* grid = nullptr;
    double dt = 0.0;
    int64_t steps_total = 0, steps_done = 0;
    double l2 = 0.0, linf = 0.0;
    int err = NR_OK;           // the status that ended a failed request
    // host-side set-up computed ahead by the server's worker: 0 none, 1 asked for, 2 being computed,
    // 3 ready (setup_rc: its status)
    int setup_state = 0;
    int setup_rc = NR_OK;
    std::unique_ptr<nrk::HostSetup> setup;
    uint64_t digest = 0;
    bool has_digest = false;
    std::vector<double> state;
};

size_t grid_bytes_estimate(const int N[3], int NG)
{
    const size_t T = (size_t)(N[0] + 2 * NG) * (N[1] + 2 * NG) * (N[2] + 2 * NG);
    // four 24-gridfunction sets, two sets of stored first differences (11 gridfunctions
    // each), maps and lists (generous per-point allowance)
    return T * (4 * 24 * sizeof(double) + 2 * 11 * sizeof(double) + 64);
}

}  // namespace

struct nr_server {
    size_t budget = 0;
    int max_slots = 0;
    int device = 0;
    void* stream = nullptr;
    int64_t next_id = 1;
    std::deque<Request*> queue;
    std::vector<Request*> running;   // resident: grid allocated, not finished
    std::vector<Request*> active;    // the running requests the batches advance
    std::map<int64_t, Request*> all;
    // one batch per kind of grid among the active requests (coordinate family x azimuth kind)
    std::vector<nr_batch*> batches;
    std::vector<std::vector<Request*>> groups;
    bool batch_dirty = true;
    size_t used = 0;
    int tile_x = 0, tile_y = 0;   // 0: autotune on every rebuild
    int policy = NR_SERVE_FIFO;
    double max_starve_s = 0.0;    // SRPT: requests submitted longer ago than this go first (0: off)
    int64_t max_points = 0;       // 0: no cap on the interior points advanced together
    // at most one chunk queued behind the running one, so that a new arrival
    // is scheduled within about a chunk of GPU time
    cudaEvent_t chunk_done[2] = {nullptr, nullptr};
    bool chunk_pending[2] = {false, false};
    int chunk_slot = 0;
    // non-finite guard: every guard_every steps (0: off) one k_finite per advanced request
    // into dflags, copied to hflags (pinned) behind the chunk; read when the chunk's event is
    // waited for, i.e. one chunk later
    int guard_every = 100;
    int64_t since_guard = 0;
    int* dflags = nullptr;          // 2 * max_slots ints on the device
    int* hflags = nullptr;          // 2 * max_slots ints, pinned host
    std::vector<int64_t> checked[2];   // ids of the requests checked behind each chunk slot
    // the set-up worker: computes HostSetup for the requests in prep_jobs (under mu)
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> prep_jobs;
    bool stop = false;
    // 0: a request's host-side set-up is computed when it is admitted; k > 0: the set-ups of the
    // next k queued requests (in admission order) are computed ahead by the worker thread, and a
    // request waits in the queue until its set-up is ready unless nothing runs
    int prefetch = 0;
    // host-side accounting (nr_server_stats): chunks, batch rebuilds, admissions, retirements;
    // seconds in admission, retirement, batch rebuilds, waits at chunk fences, enqueueing chunks
    int64_t n_chunks = 0, n_rebuilds = 0, n_admitted = 0, n_retired = 0;
    double t_admit = 0.0, t_retire = 0.0, t_rebuild = 0.0, t_fence = 0.0, t_enqueue = 0.0;
};

namespace {

void drop_batch(nr_server* s)
{
    for (nr_batch* b : s->batches) nr_batch_destroy(b);
    s->batches.clear();
    s->groups.clear();
    s->batch_dirty = true;
}

// After a chunk has been enqueued: mark its end, then wait for the chunk
// before it, which bounds the work queued ahead of the scheduler.
int chunk_fence(nr_server* s)
{
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 2 && e == cudaSuccess; q++)
        if (!s->chunk_done[q]) e = cudaEventCreateWithFlags(&s->chunk_done[q], cudaEventDisableTiming);
    const int me = s->chunk_slot, other = 1 - s->chunk_slot;
    if (e == cudaSuccess) e = cudaEventRecord(s->chunk_done[me], (cudaStream_t)s->stream);
    if (e == cudaSuccess) s->chunk_pending[me] = true;
    if (e == cudaSuccess && s->chunk_pending[other]) {
        e = cudaEventSynchronize(s->chunk_done[other]);
        s->chunk_pending[other] = false;
    }
    s->chunk_slot = other;
    cudaSetDevice(prev);
    return e == cudaSuccess ? NR_OK : nrk_fail(NR_ECUDA, "server chunk fence: %s", cudaGetErrorString(e));
}

// Enqueue the non-finite guard of the requests the current chunk advanced, behind that chunk
// (before its fence records the chunk's event), into the flags of the current chunk slot.
int guard_enqueue(nr_server* s)
{
    const int slot = s->chunk_slot;
    s->checked[slot].clear();
    if (s->guard_every <= 0 || s->since_guard < s->guard_every || s->active.empty()) return NR_OK;
    s->since_guard = 0;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaError_t e = cudaSuccess;
    if (!s->dflags) {
        e = cudaMalloc(&s->dflags, sizeof(int) * 2 * (size_t)s->max_slots);
        if (e == cudaSuccess) e = cudaMallocHost(&s->hflags, sizeof(int) * 2 * (size_t)s->max_slots);
    }
    int* d = s->dflags + (size_t)slot * s->max_slots;
    int* h = s->hflags + (size_t)slot * s->max_slots;
    const cudaStream_t st = (cudaStream_t)s->stream;
    const int n = (int)s->active.size();
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int) * n, st);
    for (int q = 0; q < n && e == cudaSuccess; q++) {
        nr_grid* g = s->active[q]->grid;
        e = nrk::launch_finite(g->K, g->y, d + q, st);
        s->checked[slot].push_back(s->active[q]->id);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        s->checked[slot].clear();
        return nrk_fail(NR_ECUDA, "server guard: %s", cudaGetErrorString(e));
    }
    return NR_OK;
}

// requests that can share one batch: same coordinate family, azimuth kind, order and integrator
int request_kind(const Request* r)
{
    const nr_grid* g = r->grid;
    return 8 * r->P.integrator + 4 * (g->K.ord == 8) + 2 * g->K.fam + (g->K.ax >= 0 ? 1 : 0);
}

void worker_loop(nr_server* s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] { return s->stop || !s->prep_jobs.empty(); });
        if (s->stop) return;
        Request* r = s->prep_jobs.front();
        s->prep_jobs.pop_front();
        if (r->setup_state != 1) continue;
        r->setup_state = 2;
        nr_params P = r->P;
        P.device = s->device;
        P.stream = s->stream;
        lk.unlock();
        std::unique_ptr<nrk::HostSetup> H(new nrk::HostSetup());
        int rc;
        try {
            rc = nrk::host_setup(r->coords, r->N, P, *H);
        } catch (...) {
            rc = NR_ENOMEM;
        }
        lk.lock();
        r->setup = std::move(H);
        r->setup_rc = rc;
        r->setup_state = 3;
        s->cv.notify_all();
    }
}

// ask the worker for the set-up of the next queued requests in admission order
void prefetch_setups(nr_server* s);

int start_request(nr_server* s, Request* r)
{
    nr_params P = r->P;
    P.device = s->device;
    P.stream = s->stream;
    std::unique_ptr<nrk::HostSetup> H;
    int rc = NR_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (r->setup_state == 1) {   // asked for, not started: computed here instead
            r->setup_state = 0;
        } else if (r->setup_state >= 2) {
            s->cv.wait(lk, [&] { return r->setup_state == 3; });
            H = std::move(r->setup);
            rc = r->setup_rc;
            r->setup_state = 0;
        }
    }
    if (!H) {
        H.reset(new nrk::HostSetup());
        rc = nrk::host_setup(r->coords, r->N, P, *H);
    }
    if (rc == NR_OK) rc = nrk::grid_from_setup(*H, P, &r->grid);
    H.reset();
    if (rc) return rc;
    rc = nr_set_brill_lindquist(r->grid, r->np, r->mass, r->xyz, 0.0, 0);
    if (rc) {
        nr_grid_destroy(r->grid);
        r->grid = nullptr;
        return rc;
    }
    r->dt = r->grid->dt_cfl;
    r->steps_total = (int64_t)ceil(r->t_final / r->dt - 1e-9);
    if (r->steps_total < 1) r->steps_total = 1;
    r->steps_done = 0;
    r->status = 1;
    return NR_OK;
}

int finish_request(nr_server* s, Request* r)
{
    int rc = nr_hamiltonian(r->grid, nullptr, nullptr, &r->l2, &r->linf);
    if (rc == NR_OK && (r->keep_state & 1)) {
        r->state.resize((size_t)NR_NGF * r->grid->geo.T);
        rc = nr_get_state(r->grid, r->state.data(), 1);
    }
    if (rc == NR_OK && (r->keep_state & 2)) {
        rc = nr_state_digest(r->grid, nullptr, &r->digest);
        r->has_digest = rc == NR_OK;
    }
    if (rc == NR_OK && nr_check_finite(r->grid) != NR_OK) rc = NR_ENONFINITE;
    r->status = rc == NR_OK ? 2 : 3;
    r->err = rc;
    if (rc != NR_OK) r->state.clear();
    nr_grid_destroy(r->grid);
    r->grid = nullptr;
    s->used -= std::min(s->used, r->bytes);
    return NR_OK;
}

// a running request the guard found non-finite: retired as failed, nothing kept
void fail_request(nr_server* s, Request* r)
{
    r->status = 3;
    r->err = NR_ENONFINITE;
    r->l2 = r->linf = NAN;
    nr_grid_destroy(r->grid);
    r->grid = nullptr;
    s->used -= std::min(s->used, r->bytes);
}

// right-hand-side evaluations per step
int64_t substeps(const Request* r) { return r->P.integrator == NR_SSPRK3 ? 3 : 4; }

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// work left, in point-substeps (a queued request: all of it, from its CFL step)
int64_t work_left(const Request* r)
{
    const int64_t steps = r->status == 0 ? r->steps_est : r->steps_total - r->steps_done;
    return steps * r->interior * substeps(r);
}

// the policy's order.  FIFO: arrival (id).  SRPT: least work left first, ties by arrival; with a
// starvation cap, requests submitted more than max_starve_s ago come first, in arrival order.
bool policy_before(const nr_server* s, const Request* a, const Request* b, double now)
{
    if (s->policy != NR_SERVE_SRPT) return a->id < b->id;
    if (s->max_starve_s > 0.0) {
        const bool sa = now - a->submit_t > s->max_starve_s, sb = now - b->submit_t > s->max_starve_s;
        if (sa != sb) return sa;
        if (sa) return a->id < b->id;
    }
    const int64_t wa = work_left(a), wb = work_left(b);
    return wa != wb ? wa < wb : a->id < b->id;
}

// make queued requests resident, in policy order, while budget and slots allow
int admit(nr_server* s)
{
    prefetch_setups(s);
    bool progress = true;
    while (!s->queue.empty() && progress) {
        progress = false;
        std::vector<Request*> order(s->queue.begin(), s->queue.end());
        const double now = now_s();
        std::sort(order.begin(), order.end(),
                  [&](const Request* a, const Request* b) { return policy_before(s, a, b, now); });
        for (Request* r : order) {
            if ((int)s->running.size() >= s->max_slots) break;
            const size_t pos = (size_t)(std::find(s->queue.begin(), s->queue.end(), r) - s->queue.begin());
            if (s->used + r->bytes > s->budget) {
                if (s->running.empty()) {   // can never fit
                    r->status = 3;
                    r->err = NR_ENOMEM;
                    s->queue.erase(s->queue.begin() + pos);
                    progress = true;
                    break;
                }
                break;   // the policy's next request waits for memory
            }
            if (s->prefetch > 0 && !s->running.empty()) {
                std::lock_guard<std::mutex> lk(s->mu);
                if (r->setup_state != 3) continue;   // set-up not ready: admitted later, the GPU is busy
            }
            s->queue.erase(s->queue.begin() + pos);
            const double t0 = now_s();
            const int rc = start_request(s, r);
            s->t_admit += now_s() - t0;
            s->n_admitted++;
            if (rc != NR_OK) {
                r->status = 3;
                r->err = rc;
            } else {
                s->used += r->bytes;
                s->running.push_back(r);
                s->batch_dirty = true;
            }
            progress = true;
            break;
        }
    }
    prefetch_setups(s);
    return NR_OK;
}

void prefetch_setups(nr_server* s)
{
    if (s->prefetch <= 0 || s->queue.empty()) return;
    // the admission order of the queue: policy order (next_queued picks the first of it)
    std::vector<Request*> order(s->queue.begin(), s->queue.end());
    const double now = now_s();
    std::sort(order.begin(), order.end(), [&](const Request* a, const Request* b) { return policy_before(s, a, b, now); });
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->worker.joinable()) s->worker = std::thread(worker_loop, s);
    int k = 0;
    for (Request* r : order) {
        if (k++ >= s->prefetch) break;
        if (r->setup_state != 0) continue;
        r->setup_state = 1;
        s->prep_jobs.push_back(r);
    }
    s->cv.notify_all();
}

// the running requests the next chunk advances: the longest prefix of the
// policy order within the points cap (never empty while any request runs)
void select_active(nr_server* s)
{
    std::vector<Request*> order = s->running;
    const double now = now_s();
    std::sort(order.begin(), order.end(), [&](const Request* a, const Request* b) { return policy_before(s, a, b, now); });
    std::vector<Request*> sel;
    int64_t pts = 0;
    for (Request* r : order) {
        if (!sel.empty() && s->max_points > 0 && pts + r->interior > s->max_points) break;
        sel.push_back(r);
        pts += r->interior;
    }
    if (sel != s->active) {
        s->active = sel;
        s->batch_dirty = true;
    }
}

int rebuild_batch(nr_server* s)
{
    drop_batch(s);
    if (s->active.empty()) return NR_OK;
    std::map<int, size_t> slot;
    for (Request* r : s->active) {
        const int k = request_kind(r);
        auto it = slot.find(k);
        if (it == slot.end()) {
            it = slot.emplace(k, s->groups.size()).first;
            s->groups.emplace_back();
        }
        s->groups[it->second].push_back(r);
    }
    for (const auto& grp : s->groups) {
        std::vector<nr_grid*> g;
        std::vector<double> dts;
        for (Request* r : grp) {
            g.push_back(r->grid);
            dts.push_back(r->dt);
        }
        nr_batch* b = nullptr;
        int rc = nr_batch_create(g.data(), (int)g.size(), &b);
        if (rc) return rc;
        s->batches.push_back(b);
        if (s->tile_x > 0)
            rc = nr_batch_set_tile(b, s->tile_x, s->tile_y);
        else
            rc = nr_batch_autotune(b, dts.data(), nullptr, nullptr, nullptr);
        if (rc) return rc;
    }
    s->batch_dirty = false;
    return NR_OK;
}

}  // namespace

extern "C" {

static int nr_server_create_body(size_t hbm_budget_bytes, int max_slots, int device, void* stream, nr_server** out)
{
    if (!out || max_slots < 1 || hbm_budget_bytes == 0) return nrk_fail(NR_EINVAL, "bad nr_server_create arguments");
    nr_server* s = new nr_server();
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->device = device;
    s->stream = stream;
    *out = s;
    return NR_OK;
}

int nr_server_create(size_t hbm_budget_bytes, int max_slots, int device, void* stream, nr_server** out)
{
    return nrk_guard("nr_server_create",
                     [&] { return nr_server_create_body(hbm_budget_bytes, max_slots, device, stream, out); });
}

void nr_server_destroy(nr_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->prep_jobs.clear();
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    drop_batch(s);
    for (int q = 0; q < 2; q++)
        if (s->chunk_done[q]) cudaEventDestroy(s->chunk_done[q]);
    if (s->dflags) cudaFree(s->dflags);
    if (s->hflags) cudaFreeHost(s->hflags);
    for (auto& kv : s->all) {
        if (kv.second->grid) nr_grid_destroy(kv.second->grid);
        delete kv.second;
    }
    delete s;
}

int nr_server_set_tile(nr_server* s, int tile_x, int tile_y)
{
    if (!s) return nrk_fail(NR_EINVAL, "server is NULL");
    s->tile_x = tile_x;
    s->tile_y = tile_y;
    s->batch_dirty = true;
    return NR_OK;
}

static int nr_server_submit_body(nr_server* s, int coords, const int Nxx[3], const nr_params* params, int npunct,
                                 const double* mass, const double* xyz, double t_final, int keep_state, int64_t* id_out)
{
    if (!s || !Nxx || !params || npunct < 0 || npunct > 16 || (npunct && (!mass || !xyz)) || !(t_final > 0.0))
        return nrk_fail(NR_EINVAL, "bad nr_server_submit arguments");
    if (params->integrator != NR_RK4 && params->integrator != NR_SSPRK3)
        return nrk_fail(NR_EINVAL, "unknown integrator %d", params->integrator);
    if (s->running.size() + s->queue.size() > 0 && s->all.size() > 1000000)
        return nrk_fail(NR_EINVAL, "too many requests");
    Request* r = new Request();
    r->id = s->next_id++;
    r->coords = coords;
    memcpy(r->N, Nxx, sizeof r->N);
    r->P = *params;
    r->np = npunct;
    for (int q = 0; q < npunct; q++) {
        r->mass[q] = mass[q];
        for (int d = 0; d < 3; d++) r->xyz[3 * q + d] = xyz[3 * q + d];
    }
    r->t_final = t_final;
    r->keep_state = keep_state;
    r->bytes = grid_bytes_estimate(Nxx, params->NG);
    r->interior = (int64_t)Nxx[0] * Nxx[1] * Nxx[2];
    double dt = 0.0;
    if (nr_dt_cfl(coords, Nxx, params, &dt) != NR_OK || !(dt > 0.0)) {
        delete r;
        s->next_id--;
        return nrk_fail(NR_EINVAL, "request grid has no valid CFL step");
    }
    r->steps_est = std::max<int64_t>(1, (int64_t)ceil(t_final / dt - 1e-9));
    r->submit_t = now_s();
    s->queue.push_back(r);
    s->all[r->id] = r;
    if (id_out) *id_out = r->id;
    return NR_OK;
}

int nr_server_submit(nr_server* s, int coords, const int Nxx[3], const nr_params* params, int npunct,
                     const double* mass, const double* xyz, double t_final, int keep_state, int64_t* id_out)
{
    return nrk_guard("nr_server_submit", [&] {
        return nr_server_submit_body(s, coords, Nxx, params, npunct, mass, xyz, t_final, keep_state, id_out);
    });
}

int nr_server_set_policy(nr_server* s, int policy, int64_t max_batch_points)
{
    if (!s) return nrk_fail(NR_EINVAL, "server is NULL");
    if ((policy != NR_SERVE_FIFO && policy != NR_SERVE_SRPT) || max_batch_points < 0)
        return nrk_fail(NR_EINVAL, "bad nr_server_set_policy arguments");
    s->policy = policy;
    s->max_points = max_batch_points;
    return NR_OK;
}

int nr_server_stats(const nr_server* s, double out[9])
{
    if (!s || !out) return nrk_fail(NR_EINVAL, "bad nr_server_stats arguments");
    const double v[9] = {(double)s->n_chunks, (double)s->n_rebuilds, (double)s->n_admitted, (double)s->n_retired,
                         s->t_admit, s->t_retire, s->t_rebuild, s->t_fence, s->t_enqueue};
    memcpy(out, v, sizeof v);
    return NR_OK;
}

int nr_server_set_starvation_cap(nr_server* s, double seconds)
{
    if (!s || !(seconds >= 0.0)) return nrk_fail(NR_EINVAL, "bad nr_server_set_starvation_cap arguments");
    s->max_starve_s = seconds;
    return NR_OK;
}

int nr_server_set_prefetch(nr_server* s, int depth)
{
    if (!s || depth < 0) return nrk_fail(NR_EINVAL, "bad nr_server_set_prefetch arguments");
    s->prefetch = depth;
    return NR_OK;
}

int nr_server_set_guard(nr_server* s, int every_steps)
{
    if (!s || every_steps < 0) return nrk_fail(NR_EINVAL, "bad nr_server_set_guard arguments");
    s->guard_every = every_steps;
    return NR_OK;
}

static int nr_server_advance_body(nr_server* s, int nsteps, int* n_running, int* n_queued)
{
    if (!s || nsteps < 0) return nrk_fail(NR_EINVAL, "bad nr_server_advance arguments");
    int rc = admit(s);
    int left = nsteps;
    while (left > 0 && !s->running.empty()) {
        select_active(s);
        if (s->batch_dirty) {
            const double t0 = now_s();
            rc = rebuild_batch(s);
            s->t_rebuild += now_s() - t0;
            s->n_rebuilds++;
            if (rc) return rc;
        }
        const double te = now_s();
        int64_t k = left;
        for (Request* r : s->active) k = std::min(k, r->steps_total - r->steps_done);
        for (size_t q = 0; q < s->batches.size(); q++) {
            std::vector<double> dts;
            for (Request* r : s->groups[q]) dts.push_back(r->dt);
            rc = s->groups[q][0]->P.integrator == NR_SSPRK3 ? nr_batch_ssprk3_step(s->batches[q], dts.data(), (int)k)
                                                             : nr_batch_rk4_step(s->batches[q], dts.data(), (int)k);
            if (rc) return rc;
        }
        for (Request* r : s->active) r->steps_done += k;
        s->since_guard += k;
        if ((rc = guard_enqueue(s))) return rc;
        const double tf = now_s();
        s->t_enqueue += tf - te;
        s->n_chunks++;
        if ((rc = chunk_fence(s))) return rc;
        s->t_fence += now_s() - tf;
        left -= (int)k;
        bool retired = false;
        // the guard results of the chunk the fence waited for (the slot it leaves current)
        std::vector<int64_t> bad;
        {
            const int slot = s->chunk_slot;
            const int* h = s->hflags ? s->hflags + (size_t)slot * s->max_slots : nullptr;
            for (size_t q = 0; q < s->checked[slot].size(); q++)
                if (h[q]) bad.push_back(s->checked[slot][q]);
            s->checked[slot].clear();
        }
        if (!bad.empty()) {
            // the queued chunk may still use the failing grids: drain the stream first
            int prev = 0;
            cudaGetDevice(&prev);
            cudaSetDevice(s->device);
            cudaError_t e = cudaStreamSynchronize((cudaStream_t)s->stream);
            cudaSetDevice(prev);
            if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "server: %s", cudaGetErrorString(e));
            s->chunk_pending[0] = s->chunk_pending[1] = false;
            s->checked[0].clear();
            s->checked[1].clear();
        }
        for (size_t q = 0; q < s->running.size();) {
            Request* r = s->running[q];
            const bool failed = std::find(bad.begin(), bad.end(), r->id) != bad.end();
            if (failed || r->steps_done >= r->steps_total) {
                if (!retired) {
                    drop_batch(s);  // the batch refers to the grids about to be released
                    retired = true;
                }
                const double t0 = now_s();
                if (failed)
                    fail_request(s, r);
                else
                    finish_request(s, r);
                s->t_retire += now_s() - t0;
                s->n_retired++;
                s->running.erase(s->running.begin() + q);
            } else {
                q++;
            }
        }
        if (retired) {
            s->active.clear();
            s->batch_dirty = true;
            admit(s);
        }
    }
    if (n_running) *n_running = (int)s->running.size();
    if (n_queued) *n_queued = (int)s->queue.size();
    return NR_OK;
}

int nr_server_advance(nr_server* s, int nsteps, int* n_running, int* n_queued)
{
    return nrk_guard("nr_server_advance", [&] { return nr_server_advance_body(s, nsteps, n_running, n_queued); });
}

int nr_server_poll(nr_server* s, int64_t id, int* status, int64_t* steps_done, int64_t* steps_total, double* l2,
                   double* linf)
{
    if (!s) return nrk_fail(NR_EINVAL, "server is NULL");
    auto it = s->all.find(id);
    if (it == s->all.end()) return nrk_fail(NR_EINVAL, "unknown request %lld", (long long)id);
    const Request* r = it->second;
    if (status) *status = r->status;
    if (steps_done) *steps_done = r->steps_done;
    if (steps_total) *steps_total = r->steps_total;
    if (l2) *l2 = r->l2;
    if (linf) *linf = r->linf;
    return NR_OK;
}

static int nr_server_fetch_state_body(nr_server* s, int64_t id, double* host_state, size_t capacity_doubles)
{
    if (!s || !host_state) return nrk_fail(NR_EINVAL, "bad nr_server_fetch_state arguments");
    auto it = s->all.find(id);
    if (it == s->all.end()) return nrk_fail(NR_EINVAL, "unknown request %lld", (long long)id);
    Request* r = it->second;
    if (r->status != 2 || r->state.empty()) return nrk_fail(NR_EINVAL, "request %lld has no kept state", (long long)id);
    if (capacity_doubles < r->state.size()) return nrk_fail(NR_EINVAL, "buffer too small");
    memcpy(host_state, r->state.data(), sizeof(double) * r->state.size());
    return NR_OK;
}

int nr_server_fetch_state(nr_server* s, int64_t id, double* host_state, size_t capacity_doubles)
{
    return nrk_guard("nr_server_fetch_state",
                     [&] { return nr_server_fetch_state_body(s, id, host_state, capacity_doubles); });
}

int nr_server_fetch_digest(nr_server* s, int64_t id, uint64_t* digest)
{
    if (!s || !digest) return nrk_fail(NR_EINVAL, "bad nr_server_fetch_digest arguments");
    auto it = s->all.find(id);
    if (it == s->all.end()) return nrk_fail(NR_EINVAL, "unknown request %lld", (long long)id);
    const Request* r = it->second;
    if (r->status != 2 || !r->has_digest) return nrk_fail(NR_EINVAL, "request %lld has no kept digest", (long long)id);
    *digest = r->digest;
    return NR_OK;
}

int nr_server_request_error(nr_server* s, int64_t id, int* code)
{
    if (!s || !code) return nrk_fail(NR_EINVAL, "bad nr_server_request_error arguments");
    auto it = s->all.find(id);
    if (it == s->all.end()) return nrk_fail(NR_EINVAL, "unknown request %lld", (long long)id);
    *code = it->second->err;
    return NR_OK;
}

}  // extern "C"
