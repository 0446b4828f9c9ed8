// nr_part.cu -- one grid split into partitions (the chare decomposition of Sec. 3).
//
// The interior of the padded grid is cut along each axis into parts[d] slabs of
// nearly equal size, each at least N_G points thick.  A partition owns its
// interior box and, at the edges of the grid, the ghost layers beyond it; it
// stores that box widened by N_G on every side (its halo).  After every
// integrator substage:
//   1. every partition computes the right-hand side and the stage update at the
//      interior and pure-outer points it owns (the single-grid kernels, on a
//      GridK that describes the partition's box);
//   2. inner (parity) boundary points are filled from their sources -- within a
//      partition by the parity-copy kernel, across partitions by messages built
//      at set-up from the boundary map, as the paper's per-chare send lists of
//      remote inner-boundary points;
//   3. halos are exchanged face by face in the paper's order, along axis 0, then
//      axis 1, then axis 2 (E-W, N-S, T-B); each phase sends the slab of width
//      N_G next to a face, spanning the halos already filled along earlier axes,
//      so edge and corner halos arrive without diagonal messages.
// A message gathers its values on the sending partition into a send buffer
// (k_pack), is copied into the receiving partition's buffer (cudaMemcpyAsync,
// the transfer), and is scattered there with its parity signs (k_unpack).  All
// partitions of a grid live on one device here, so the transfer is a
// device-local copy; every point runs the single-grid arithmetic on the same
// values, so the partitioned evolution is bitwise that of the whole grid.
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "nr_internal.h"
#include "nr_stage.cuh"

namespace nrk {

// ------------------------------------------------------------------ plan

struct PartBox {
    int q[3];
    int lo[3], hi[3];     // interior range, global padded indices
    int olo[3], ohi[3];   // owned range (ghost layers included at the grid's edges)
    int org[3];           // local origin: lo - NG
    int m[3];             // local padded sizes: hi - lo + 2 NG
    long T;
    long local(int g0, int g1, int g2) const
    {
        return (g0 - org[0]) + (long)m[0] * ((g1 - org[1]) + (long)m[1] * (g2 - org[2]));
    }
};

struct PartMsg {
    int src = 0, dst = 0;
    std::vector<int> sidx, didx, neg;   // neg: parity masks (phase 0 only)
};

struct PartPlan {
    int parts[3] = {1, 1, 1};
    int np = 1;
    std::vector<PartBox> box;
    std::vector<std::vector<InnerPt>> inner;   // parity copies within one partition (local indices)
    std::vector<std::vector<OuterPt>> outer;   // owned pure-outer points (local indices)
    std::vector<std::vector<int>> canon_l, canon_g;   // owned canonical points: local, global flat index
    std::vector<PartMsg> msg[4];   // 0: parity copies across partitions; 1..3: halos along axes 0, 1, 2
};

namespace {

int owner_along(const std::vector<int>& cut, int g)
{
    const int P = (int)cut.size() - 1;
    int k = (int)(std::upper_bound(cut.begin(), cut.end(), g) - cut.begin()) - 1;
    return std::min(std::max(k, 0), P - 1);
}

}  // namespace

int part_plan(const HostSetup& H, const int parts[3], PartPlan& plan)
{
    const HostGeom& G = H.G;
    const int NG = G.NG;
    long np = 1;
    for (int d = 0; d < 3; d++) {
        if (parts[d] < 1 || parts[d] > G.N[d]) return nrk_fail(NR_EINVAL, "parts[%d] = %d out of range", d, parts[d]);
        np *= parts[d];
    }
    if (np > 4096) return nrk_fail(NR_EINVAL, "%ld partitions: at most 4096", np);
    std::vector<int> cut[3];
    for (int d = 0; d < 3; d++) {
        for (int k = 0; k <= parts[d]; k++) cut[d].push_back(NG + (int)(((long)k * G.N[d]) / parts[d]));
        if (parts[d] > 1)
            for (int k = 0; k < parts[d]; k++)
                if (cut[d][k + 1] - cut[d][k] < NG)
                    return nrk_fail(NR_EINVAL, "a partition along axis %d would hold %d interior points, fewer than N_G = %d",
                                    d, cut[d][k + 1] - cut[d][k], NG);
    }
    for (int d = 0; d < 3; d++) plan.parts[d] = parts[d];
    plan.np = (int)np;
    plan.box.assign(np, PartBox{});
    for (int q2 = 0; q2 < parts[2]; q2++)
        for (int q1 = 0; q1 < parts[1]; q1++)
            for (int q0 = 0; q0 < parts[0]; q0++) {
                const int q = q0 + parts[0] * (q1 + parts[1] * q2);
                PartBox& b = plan.box[q];
                const int qq[3] = {q0, q1, q2};
                b.T = 1;
                for (int d = 0; d < 3; d++) {
                    b.q[d] = qq[d];
                    b.lo[d] = cut[d][qq[d]];
                    b.hi[d] = cut[d][qq[d] + 1];
                    b.olo[d] = qq[d] == 0 ? 0 : b.lo[d];
                    b.ohi[d] = qq[d] == parts[d] - 1 ? G.n[d] : b.hi[d];
                    b.org[d] = b.lo[d] - NG;
                    b.m[d] = b.hi[d] - b.lo[d] + 2 * NG;
                    b.T *= b.m[d];
                }
            }
    const int n0 = G.n[0], n1 = G.n[1];
    auto coords_of = [&](long idx, int g[3]) {
        g[0] = (int)(idx % n0);
        g[1] = (int)((idx / n0) % n1);
        g[2] = (int)(idx / ((long)n0 * n1));
    };
    auto owner = [&](const int g[3]) {
        return owner_along(cut[0], g[0]) + parts[0] * (owner_along(cut[1], g[1]) + parts[1] * owner_along(cut[2], g[2]));
    };
    plan.inner.assign(np, {});
    plan.outer.assign(np, {});
    plan.canon_l.assign(np, {});
    plan.canon_g.assign(np, {});
    for (int ph = 0; ph < 4; ph++) plan.msg[ph].clear();
    for (const OuterPt& o : H.outer) {
        int g[3];
        coords_of(o.idx, g);
        const int q = owner(g);
        OuterPt l = o;
        l.idx = (int)plan.box[q].local(g[0], g[1], g[2]);
        plan.outer[q].push_back(l);
    }
    for (int idx : H.canon) {
        int g[3];
        coords_of(idx, g);
        const int q = owner(g);
        plan.canon_l[q].push_back((int)plan.box[q].local(g[0], g[1], g[2]));
        plan.canon_g[q].push_back(idx);
    }
    // inner boundary: a copy within the partition, or a message from the source's owner
    std::map<std::pair<int, int>, size_t> slot;
    for (const InnerPt& p : H.inner) {
        int gd[3], gs[3];
        coords_of(p.dst, gd);
        coords_of(p.src, gs);
        const int qd = owner(gd), qs = owner(gs);
        const int dl = (int)plan.box[qd].local(gd[0], gd[1], gd[2]);
        const int sl = (int)plan.box[qs].local(gs[0], gs[1], gs[2]);
        if (qd == qs) {
            plan.inner[qd].push_back(InnerPt{dl, sl, p.negmask, 0});
            continue;
        }
        auto it = slot.find({qs, qd});
        if (it == slot.end()) {
            it = slot.emplace(std::make_pair(qs, qd), plan.msg[0].size()).first;
            plan.msg[0].emplace_back();
            plan.msg[0].back().src = qs;
            plan.msg[0].back().dst = qd;
        }
        PartMsg& m = plan.msg[0][it->second];
        m.sidx.push_back(sl);
        m.didx.push_back(dl);
        m.neg.push_back(p.negmask);
    }
    // halos, face by face: phase 1 + d fills the halo of width NG along axis d, spanning the
    // local box along earlier axes and the owned range along later ones
    for (int d = 0; d < 3; d++) {
        if (parts[d] == 1) continue;
        for (int q = 0; q < (int)np; q++) {
            const PartBox& b = plan.box[q];
            for (int side = 0; side < 2; side++) {
                if (side == 0 && b.q[d] == 0) continue;
                if (side == 1 && b.q[d] == parts[d] - 1) continue;
                int qn[3] = {b.q[0], b.q[1], b.q[2]};
                qn[d] += side == 0 ? -1 : 1;
                const int qs = qn[0] + parts[0] * (qn[1] + parts[1] * qn[2]);
                const PartBox& s = plan.box[qs];
                int r0[3], r1[3];
                for (int e = 0; e < 3; e++) {
                    if (e == d) {
                        r0[e] = side == 0 ? b.lo[d] - NG : b.hi[d];
                        r1[e] = side == 0 ? b.lo[d] : b.hi[d] + NG;
                    } else if (e < d) {
                        r0[e] = b.org[e];
                        r1[e] = b.org[e] + b.m[e];
                    } else {
                        r0[e] = b.olo[e];
                        r1[e] = b.ohi[e];
                    }
                }
                PartMsg m;
                m.src = qs;
                m.dst = q;
                for (int g2 = r0[2]; g2 < r1[2]; g2++)
                    for (int g1 = r0[1]; g1 < r1[1]; g1++)
                        for (int g0 = r0[0]; g0 < r1[0]; g0++) {
                            m.sidx.push_back((int)s.local(g0, g1, g2));
                            m.didx.push_back((int)b.local(g0, g1, g2));
                        }
                plan.msg[1 + d].push_back(std::move(m));
            }
        }
    }
    return NR_OK;
}

// ---------------------------------------------------------------- kernels

// send buffer of a message: buf[g n + t] = y[g T + idx[t]]
__global__ void __launch_bounds__(256) k_pack(long T, const int* __restrict__ idx, int n, const double* __restrict__ y,
                                              double* __restrict__ buf)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int g = blockIdx.y;
    buf[(long)g * n + t] = y[(long)g * T + idx[t]];
}

// receive side: y[g T + idx[t]] = p buf[g n + t], the parity sign p of gridfunction g's tensor type
// (mask bit set: -1) applied to the bit pattern
__global__ void __launch_bounds__(256) k_unpack(long T, const int* __restrict__ idx, const int* __restrict__ neg, int n,
                                                const double* __restrict__ buf, double* __restrict__ y)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int g = blockIdx.y;
    long long v = __double_as_longlong(buf[(long)g * n + t]);
    if (neg) v ^= (long long)((neg[t] >> gf_type(g)) & 1) << 63;
    y[(long)g * T + idx[t]] = __longlong_as_double(v);
}

// a partition's box to or from a 24-gridfunction set of the whole grid (n: its padded sizes):
// to_part copies every point of the box, otherwise only the owned points are written back
__global__ void __launch_bounds__(256) k_box(long Tg, int n0, int n1, PartBox b, bool to_part, double* __restrict__ whole,
                                             double* __restrict__ part)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.T) return;
    const int l0 = (int)(t % b.m[0]), l1 = (int)((t / b.m[0]) % b.m[1]), l2 = (int)(t / ((long)b.m[0] * b.m[1]));
    const int g0 = l0 + b.org[0], g1 = l1 + b.org[1], g2 = l2 + b.org[2];
    const long gi = g0 + (long)n0 * (g1 + (long)n1 * g2);
    const int g = blockIdx.y;
    if (to_part) {
        part[(long)g * b.T + t] = whole[(long)g * Tg + gi];
    } else if (g0 >= b.olo[0] && g0 < b.ohi[0] && g1 >= b.olo[1] && g1 < b.ohi[1] && g2 >= b.olo[2] &&
               g2 < b.ohi[2]) {
        whole[(long)g * Tg + gi] = part[(long)g * b.T + t];
    }
}

struct DevMsg {
    int src = 0, dst = 0, n = 0;
    int *sidx = nullptr, *didx = nullptr, *neg = nullptr;
    double *sbuf = nullptr, *rbuf = nullptr;
};

struct PartDev {
    PartBox b;
    GridK K;
    double *y = nullptr, *ya = nullptr, *yb = nullptr, *acc = nullptr, *d1x = nullptr, *d1y = nullptr;
    double *ax0 = nullptr, *ax1 = nullptr, *ax2 = nullptr;
    OuterPt* outer = nullptr;
    int n_outer = 0;
    InnerPt* inner = nullptr;
    int n_inner = 0;
    int *canon = nullptr, *canon_g = nullptr;
    long n_canon = 0;
};

}  // namespace nrk

using namespace nrk;

struct nr_part {
    nr_params P;
    HostGeom G;
    GridK K;   // the whole grid's kernel description (no device arrays)
    double dt_cfl = 0.0;
    int parts[3] = {1, 1, 1};
    int device = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    // per-partition streams and events: inside the captured step each partition's kernels form their
    // own branch of the graph, so the partitions' launches overlap on the GPU
    std::vector<cudaStream_t> pstream;
    std::vector<cudaEvent_t> pevent;
    cudaEvent_t fork = nullptr;
    std::vector<PartDev> p;
    std::vector<DevMsg> msg[4];
    double* finf = nullptr;
    double* wspeed = nullptr;
    double* mxyz = nullptr;
    double* whole = nullptr;   // staging of a whole-grid state (nr_part_set_state / get_state), on first use
    // constraint norms: every partition's block partials side by side, one fixed-order reduction
    double* partials = nullptr;
    std::vector<int> part_off;   // first partial of each partition
    int nparts_total = 0;
    double* hres = nullptr;
    unsigned long long* digest = nullptr;
    std::vector<double> cart_canon;
    cudaGraphExec_t exec = nullptr;
    double graph_dt = 0.0;
    int graph_kind = -1;
    size_t bytes = 0;
};

namespace {

struct DevGuardP {
    int prev = 0;
    explicit DevGuardP(int d) { cudaGetDevice(&prev); cudaSetDevice(d); }
    ~DevGuardP() { cudaSetDevice(prev); }
};

#define PCUDA(call)                                                                                    \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return nrk_fail(NR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

template <typename T>
int pmalloc(nr_part* s, T** ptr, size_t count)
{
    const size_t b = sizeof(T) * std::max<size_t>(count, 1);
    cudaError_t e = cudaMalloc((void**)ptr, b);
    if (e != cudaSuccess) return nrk_fail(NR_ENOMEM, "cudaMalloc(%zu): %s", b, cudaGetErrorString(e));
    s->bytes += b;
    return NR_OK;
}

template <typename T>
int pupload(nr_part* s, T** ptr, const std::vector<T>& h)
{
    int rc = pmalloc(s, ptr, h.size());
    if (rc) return rc;
    if (!h.empty()) PCUDA(cudaMemcpy(*ptr, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return NR_OK;
}

void free_part(nr_part* s)
{
    if (!s) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    for (PartDev& d : s->p) {
        void* ptrs[] = {d.y, d.ya, d.yb, d.acc, d.d1x, d.d1y, d.ax0, d.ax1, d.ax2, d.outer, d.inner, d.canon, d.canon_g};
        for (void* q : ptrs)
            if (q) cudaFree(q);
    }
    for (int ph = 0; ph < 4; ph++)
        for (DevMsg& m : s->msg[ph]) {
            void* ptrs[] = {m.sidx, m.didx, m.neg, m.sbuf, m.rbuf};
            for (void* q : ptrs)
                if (q) cudaFree(q);
        }
    void* ptrs[] = {s->finf, s->wspeed, s->mxyz, s->whole, s->digest, s->partials, s->hres};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (s->cap) cudaStreamDestroy(s->cap);
    for (cudaStream_t q : s->pstream)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : s->pevent)
        if (e) cudaEventDestroy(e);
    if (s->fork) cudaEventDestroy(s->fork);
    cudaSetDevice(prev);
    delete s;
}

// the slice [org, org + m) of each component (stride n) of a per-axis array
std::vector<double> axis_slice(const std::vector<double>& a, int n, int org, int m)
{
    const int comps = (int)(a.size() / n);
    std::vector<double> out((size_t)comps * m);
    for (int c = 0; c < comps; c++)
        for (int i = 0; i < m; i++) out[(size_t)c * m + i] = a[(size_t)c * n + org + i];
    return out;
}

// every partition's buffer of kind `which` (0 y, 1 ya, 2 yb)
double* buf_of(PartDev& d, int which) { return which == 0 ? d.y : which == 1 ? d.ya : d.yb; }

// one substage: right-hand side + stage update on every partition (input in, output out), then
// the parity copies within partitions, then the messages phase by phase
int enqueue_stage(nr_part* s, cudaStream_t st, int in, int out, const Stage& sg, bool yn_is_y, bool use_acc)
{
    // every partition's points (and its own parity copies) on its own stream, forked from and joined
    // back into st; with one partition, on st itself
    const bool forked = s->p.size() > 1 && st == s->cap;
    if (forked) PCUDA(cudaEventRecord(s->fork, st));
    for (size_t q = 0; q < s->p.size(); q++) {
        PartDev& d = s->p[q];
        cudaStream_t ps = forked ? s->pstream[q] : st;
        if (forked) PCUDA(cudaStreamWaitEvent(ps, s->fork, 0));
        OuterArgs oa;
        oa.pts = d.outer;
        oa.npts = d.n_outer;
        oa.finf = s->finf;
        oa.wspeed = s->wspeed;
        PCUDA(launch_rhs(d.K, buf_of(d, in), d.d1x, d.d1y, buf_of(d, out), yn_is_y ? d.y : nullptr,
                         use_acc ? d.acc : nullptr, sg, ps, oa));
        PCUDA(launch_inner(d.K, d.inner, d.n_inner, buf_of(d, out), ps));
        if (forked) {
            PCUDA(cudaEventRecord(s->pevent[q], ps));
            PCUDA(cudaStreamWaitEvent(st, s->pevent[q], 0));
        }
    }
    for (int ph = 0; ph < 4; ph++) {
        for (DevMsg& m : s->msg[ph]) {
            PartDev& a = s->p[m.src];
            k_pack<<<dim3((m.n + 255) / 256, NGF), 256, 0, st>>>(a.b.T, m.sidx, m.n, buf_of(a, out), m.sbuf);
            PCUDA(cudaGetLastError());
        }
        for (DevMsg& m : s->msg[ph])
            PCUDA(cudaMemcpyAsync(m.rbuf, m.sbuf, sizeof(double) * NGF * (size_t)m.n, cudaMemcpyDeviceToDevice, st));
        for (DevMsg& m : s->msg[ph]) {
            PartDev& b = s->p[m.dst];
            k_unpack<<<dim3((m.n + 255) / 256, NGF), 256, 0, st>>>(b.b.T, m.didx, m.neg, m.n, m.rbuf, buf_of(b, out));
            PCUDA(cudaGetLastError());
        }
    }
    return NR_OK;
}

// classic RK4 and SSPRK3 on the partitions, with the stage constants of the single-grid drivers
int enqueue_rk4(nr_part* s, cudaStream_t st, double dt)
{
    const int enf = s->P.enforce_detgb;
    int rc;
    if ((rc = enqueue_stage(s, st, 0, 1, Stage{MODE_STAGE1, enf, 0.5 * dt, dt / 6.0, 0.0}, true, true))) return rc;
    if ((rc = enqueue_stage(s, st, 1, 2, Stage{MODE_STAGE23, enf, 0.5 * dt, dt / 3.0, 0.0}, true, true))) return rc;
    if ((rc = enqueue_stage(s, st, 2, 1, Stage{MODE_STAGE23, enf, dt, dt / 3.0, 0.0}, true, true))) return rc;
    return enqueue_stage(s, st, 1, 0, Stage{MODE_STAGE4, enf, 0.0, dt / 6.0, 0.0}, false, true);
}

int enqueue_ssprk3(nr_part* s, cudaStream_t st, double dt)
{
    const int enf = s->P.enforce_detgb;
    int rc;
    if ((rc = enqueue_stage(s, st, 0, 1, Stage{MODE_SSP, enf, dt, 1.0, 0.0}, true, false))) return rc;
    if ((rc = enqueue_stage(s, st, 1, 2, Stage{MODE_SSP, enf, dt, 0.25, 0.75}, true, false))) return rc;
    return enqueue_stage(s, st, 2, 0, Stage{MODE_SSP, enf, dt, 2.0 / 3.0, 1.0 / 3.0}, true, false);
}

int part_steps(nr_part* s, int kind, double dt, int nsteps)
{
    if (!s || !(dt > 0.0) || nsteps < 0) return nrk_fail(NR_EINVAL, "bad partitioned step arguments");
    if (nsteps == 0) return NR_OK;
    DevGuardP dg(s->device);
    if (!s->exec || s->graph_dt != dt || s->graph_kind != kind) {
        if (s->exec) {
            cudaGraphExecDestroy(s->exec);
            s->exec = nullptr;
        }
        cudaGraph_t graph;
        PCUDA(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
        int rc = kind == NR_SSPRK3 ? enqueue_ssprk3(s, s->cap, dt) : enqueue_rk4(s, s->cap, dt);
        cudaError_t e = cudaStreamEndCapture(s->cap, &graph);
        if (rc) return rc;
        if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&s->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        s->graph_dt = dt;
        s->graph_kind = kind;
    }
    for (int n = 0; n < nsteps; n++) PCUDA(cudaGraphLaunch(s->exec, s->stream));
    return NR_OK;
}

int plan_for(int coords, const int Nxx[3], const nr_params& P, const int parts[3], HostSetup& H, PartPlan& plan)
{
    if (!parts) return nrk_fail(NR_EINVAL, "parts is NULL");
    int rc = host_setup(coords, Nxx, P, H);
    if (rc) return rc;
    return part_plan(H, parts, plan);
}

int plan_host(int coords, const int Nxx[3], int NG, const int parts[3], HostSetup& H, PartPlan& plan)
{
    nr_params P;
    nr_params_default(coords, &P);
    P.NG = NG;
    return plan_for(coords, Nxx, P, parts, H, plan);
}

}  // namespace

extern "C" {

static int nr_part_create_body(int coords, const int Nxx[3], const nr_params* params, const int parts[3], nr_part** out)
{
    if (!out) return nrk_fail(NR_EINVAL, "out is NULL");
    *out = nullptr;
    nr_params P;
    if (params)
        P = *params;
    else
        nr_params_default(coords, &P);
    HostSetup H;
    PartPlan plan;
    int rc = plan_for(coords, Nxx, P, parts, H, plan);
    if (rc) return rc;
    nr_part* s = new nr_part();
    try {
        s->P = P;
        s->G = H.G;
        s->K = H.K;
        s->dt_cfl = H.dt;
        for (int d = 0; d < 3; d++) s->parts[d] = parts[d];
        s->device = P.device;
        s->stream = (cudaStream_t)P.stream;
        s->cart_canon = H.cart_canon;
        DevGuardP dg(s->device);
        std::vector<double> finf(P.f_inf, P.f_inf + NR_NGF), ws(P.wavespeed, P.wavespeed + NR_NGF);
        if ((rc = pupload(s, &s->finf, finf)) || (rc = pupload(s, &s->wspeed, ws)) || (rc = pmalloc(s, &s->mxyz, 64)) ||
            (rc = pmalloc(s, &s->digest, 1))) {
            free_part(s);
            return rc;
        }
        s->p.resize(plan.np);
        for (int q = 0; q < plan.np; q++) {
            PartDev& d = s->p[q];
            d.b = plan.box[q];
            GridK& K = d.K;
            K = H.K;
            K.n0 = d.b.m[0]; K.n1 = d.b.m[1]; K.n2 = d.b.m[2];
            K.N0 = d.b.hi[0] - d.b.lo[0]; K.N1 = d.b.hi[1] - d.b.lo[1]; K.N2 = d.b.hi[2] - d.b.lo[2];
            K.T = d.b.T;
            const size_t set = (size_t)NR_NGF * d.b.T;
            std::vector<double> a0 = axis_slice(H.a0, H.G.n[0], d.b.org[0], d.b.m[0]);
            std::vector<double> a1 = axis_slice(H.a1, H.G.n[1], d.b.org[1], d.b.m[1]);
            std::vector<double> a2 = axis_slice(H.a2, H.G.n[2], d.b.org[2], d.b.m[2]);
            d.n_outer = (int)plan.outer[q].size();
            d.n_inner = (int)plan.inner[q].size();
            d.n_canon = (long)plan.canon_l[q].size();
            if ((rc = pmalloc(s, &d.y, set)) || (rc = pmalloc(s, &d.ya, set)) || (rc = pmalloc(s, &d.yb, set)) ||
                (rc = pmalloc(s, &d.acc, set)) || (rc = pmalloc(s, &d.d1x, (size_t)N_D1 * d.b.T)) ||
                (rc = pmalloc(s, &d.d1y, K.ax < 0 ? (size_t)N_D1 * d.b.T : 1)) || (rc = pupload(s, &d.ax0, a0)) ||
                (rc = pupload(s, &d.ax1, a1)) || (rc = pupload(s, &d.ax2, a2)) ||
                (rc = pupload(s, &d.outer, plan.outer[q])) || (rc = pupload(s, &d.inner, plan.inner[q])) ||
                (rc = pupload(s, &d.canon, plan.canon_l[q])) || (rc = pupload(s, &d.canon_g, plan.canon_g[q]))) {
                free_part(s);
                return rc;
            }
            K.rfm.ax0 = d.ax0;
            K.rfm.ax1 = d.ax1;
            K.rfm.ax2 = d.ax2;
            cudaError_t e = cudaMemset(d.y, 0, sizeof(double) * set);
            if (e == cudaSuccess) e = cudaMemset(d.acc, 0, sizeof(double) * set);
            if (e != cudaSuccess) {
                free_part(s);
                return nrk_fail(NR_ECUDA, "partition set-up: %s", cudaGetErrorString(e));
            }
        }
        s->part_off.assign(s->p.size(), 0);
        for (size_t q = 0; q < s->p.size(); q++) {
            s->part_off[q] = s->nparts_total;
            s->nparts_total += ham_partials_needed(s->p[q].K);
        }
        if ((rc = pmalloc(s, &s->partials, 3 * (size_t)s->nparts_total)) || (rc = pmalloc(s, &s->hres, 3))) {
            free_part(s);
            return rc;
        }
        for (int ph = 0; ph < 4; ph++)
            for (const PartMsg& m : plan.msg[ph]) {
                s->msg[ph].emplace_back();
                DevMsg& dm = s->msg[ph].back();
                dm.src = m.src;
                dm.dst = m.dst;
                dm.n = (int)m.sidx.size();
                if ((rc = pupload(s, &dm.sidx, m.sidx)) || (rc = pupload(s, &dm.didx, m.didx)) ||
                    (ph == 0 && (rc = pupload(s, &dm.neg, m.neg))) ||
                    (rc = pmalloc(s, &dm.sbuf, (size_t)NR_NGF * dm.n)) ||
                    (rc = pmalloc(s, &dm.rbuf, (size_t)NR_NGF * dm.n))) {
                    free_part(s);
                    return rc;
                }
            }
        cudaError_t e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming);
        s->pstream.assign(s->p.size(), nullptr);
        s->pevent.assign(s->p.size(), nullptr);
        for (size_t q = 0; q < s->p.size() && e == cudaSuccess; q++) {
            e = cudaStreamCreateWithFlags(&s->pstream[q], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->pevent[q], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = rhs_kernels_init();   // before any step is captured
        if (e != cudaSuccess) {
            free_part(s);
            return nrk_fail(NR_ECUDA, "partition streams: %s", cudaGetErrorString(e));
        }
        *out = s;
        return NR_OK;
    } catch (...) {
        free_part(s);
        throw;
    }
}

int nr_part_create(int coords, const int Nxx[3], const nr_params* params, const int parts[3], nr_part** out)
{
    return nrk_guard("nr_part_create", [&] { return nr_part_create_body(coords, Nxx, params, parts, out); });
}

void nr_part_destroy(nr_part* s) { free_part(s); }

int nr_part_query(const nr_part* s, int64_t* nparts, int64_t messages[4], double* dt_cfl, size_t* device_bytes)
{
    if (!s) return nrk_fail(NR_EINVAL, "partitioned grid is NULL");
    if (nparts) *nparts = (int64_t)s->p.size();
    if (messages)
        for (int ph = 0; ph < 4; ph++) messages[ph] = (int64_t)s->msg[ph].size();
    if (dt_cfl) *dt_cfl = s->dt_cfl;
    if (device_bytes) *device_bytes = s->bytes;
    return NR_OK;
}

static int nr_part_set_bl_body(nr_part* s, int npunct, const double* mass, const double* xyz, double perturb_amp,
                               uint64_t seed)
{
    if (!s || npunct < 0 || npunct > 16 || (npunct && (!mass || !xyz)))
        return nrk_fail(NR_EINVAL, "bad Brill-Lindquist arguments");
    for (size_t t = 0; t < s->cart_canon.size() / 3; t++)
        for (int q = 0; q < npunct; q++) {
            const double dx = s->cart_canon[3 * t] - xyz[3 * q], dy = s->cart_canon[3 * t + 1] - xyz[3 * q + 1],
                         dz = s->cart_canon[3 * t + 2] - xyz[3 * q + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) < 1e-12) return nrk_fail(NR_EINVAL, "puncture %d lies on a grid point", q);
        }
    DevGuardP dg(s->device);
    double m[64];
    for (int q = 0; q < npunct; q++) {
        m[4 * q] = mass[q];
        m[4 * q + 1] = xyz[3 * q];
        m[4 * q + 2] = xyz[3 * q + 1];
        m[4 * q + 3] = xyz[3 * q + 2];
    }
    if (npunct) PCUDA(cudaMemcpyAsync(s->mxyz, m, sizeof(double) * 4 * npunct, cudaMemcpyHostToDevice, s->stream));
    for (PartDev& d : s->p) {
        PCUDA(cudaMemsetAsync(d.y, 0, sizeof(double) * NR_NGF * d.b.T, s->stream));
        PCUDA(launch_bl(d.K, d.canon, d.n_canon, npunct, s->mxyz, perturb_amp, seed, d.y, s->stream, d.canon_g));
    }
    // the parity copies and the halos of the new state
    for (PartDev& d : s->p) PCUDA(launch_inner(d.K, d.inner, d.n_inner, d.y, s->stream));
    for (int ph = 0; ph < 4; ph++) {
        for (DevMsg& mm : s->msg[ph]) {
            PartDev& a = s->p[mm.src];
            k_pack<<<dim3((mm.n + 255) / 256, NGF), 256, 0, s->stream>>>(a.b.T, mm.sidx, mm.n, a.y, mm.sbuf);
            PCUDA(cudaGetLastError());
            PCUDA(cudaMemcpyAsync(mm.rbuf, mm.sbuf, sizeof(double) * NGF * (size_t)mm.n, cudaMemcpyDeviceToDevice,
                                  s->stream));
            PartDev& b = s->p[mm.dst];
            k_unpack<<<dim3((mm.n + 255) / 256, NGF), 256, 0, s->stream>>>(b.b.T, mm.didx, mm.neg, mm.n, mm.rbuf, b.y);
            PCUDA(cudaGetLastError());
        }
    }
    PCUDA(cudaStreamSynchronize(s->stream));
    return NR_OK;
}

int nr_part_set_brill_lindquist(nr_part* s, int npunct, const double* mass, const double* xyz, double perturb_amp,
                                uint64_t seed)
{
    return nrk_guard("nr_part_set_brill_lindquist",
                     [&] { return nr_part_set_bl_body(s, npunct, mass, xyz, perturb_amp, seed); });
}

static int part_whole(nr_part* s, double* buf, int host, bool to_part)
{
    if (!s || !buf) return nrk_fail(NR_EINVAL, "bad partitioned state arguments");
    DevGuardP dg(s->device);
    const size_t b = sizeof(double) * NR_NGF * s->G.T;
    double* whole = buf;
    if (host) {
        if (!s->whole) PCUDA(cudaMalloc(&s->whole, b));
        whole = s->whole;
        if (to_part) PCUDA(cudaMemcpyAsync(whole, buf, b, cudaMemcpyHostToDevice, s->stream));
    }
    for (PartDev& d : s->p) {
        k_box<<<dim3((unsigned)((d.b.T + 255) / 256), NGF), 256, 0, s->stream>>>(s->G.T, s->G.n[0], s->G.n[1], d.b,
                                                                                to_part, whole, d.y);
        PCUDA(cudaGetLastError());
    }
    if (host && !to_part) PCUDA(cudaMemcpyAsync(buf, whole, b, cudaMemcpyDeviceToHost, s->stream));
    if (host) PCUDA(cudaStreamSynchronize(s->stream));
    return NR_OK;
}

int nr_part_set_state(nr_part* s, const double* src, int from_host)
{
    return nrk_guard("nr_part_set_state", [&] { return part_whole(s, const_cast<double*>(src), from_host, true); });
}

int nr_part_get_state(nr_part* s, double* dst, int to_host)
{
    return nrk_guard("nr_part_get_state", [&] { return part_whole(s, dst, to_host, false); });
}

int nr_part_rk4_step(nr_part* s, double dt, int nsteps)
{
    return nrk_guard("nr_part_rk4_step", [&] { return part_steps(s, NR_RK4, dt, nsteps); });
}

int nr_part_ssprk3_step(nr_part* s, double dt, int nsteps)
{
    return nrk_guard("nr_part_ssprk3_step", [&] { return part_steps(s, NR_SSPRK3, dt, nsteps); });
}

int nr_part_digest(nr_part* s, uint64_t* out)
{
    if (!s || !out) return nrk_fail(NR_EINVAL, "bad nr_part_digest arguments");
    DevGuardP dg(s->device);
    unsigned long long total = 0;
    for (PartDev& d : s->p) {
        unsigned long long h = 0;
        PCUDA(launch_digest(d.K, d.canon, d.n_canon, d.y, s->digest, s->stream, d.canon_g));
        PCUDA(cudaMemcpyAsync(&h, s->digest, sizeof h, cudaMemcpyDeviceToHost, s->stream));
        PCUDA(cudaStreamSynchronize(s->stream));
        total += h;
    }
    *out = (uint64_t)total;
    return NR_OK;
}

static int nr_part_hamiltonian_body(nr_part* s, double* l2_out, double* linf_out)
{
    if (!s || (!l2_out && !linf_out)) return nrk_fail(NR_EINVAL, "bad nr_part_hamiltonian arguments");
    DevGuardP dg(s->device);
    // each partition's interior points into its slice of the partials (the per-partition reduction
    // it also runs writes a scratch result nobody reads), then one reduction over all of them
    for (size_t q = 0; q < s->p.size(); q++) {
        PartDev& d = s->p[q];
        PCUDA(launch_ham(d.K, d.y, nullptr, s->P.h_rmin, s->P.h_rmax, s->partials + 3 * (size_t)s->part_off[q],
                         ham_partials_needed(d.K), s->hres, s->stream));
    }
    PCUDA(launch_ham_reduce(s->partials, s->nparts_total, s->hres, s->stream));
    double r[3];
    PCUDA(cudaMemcpyAsync(r, s->hres, sizeof r, cudaMemcpyDeviceToHost, s->stream));
    PCUDA(cudaStreamSynchronize(s->stream));
    if (l2_out) *l2_out = r[0];
    if (linf_out) *linf_out = r[1];
    return NR_OK;
}

int nr_part_hamiltonian(nr_part* s, double* l2_out, double* linf_out)
{
    return nrk_guard("nr_part_hamiltonian", [&] { return nr_part_hamiltonian_body(s, l2_out, linf_out); });
}

int nr_part_sync(nr_part* s)
{
    if (!s) return nrk_fail(NR_EINVAL, "partitioned grid is NULL");
    DevGuardP dg(s->device);
    PCUDA(cudaStreamSynchronize(s->stream));
    return NR_OK;
}

// ---- host-only views of the plan

int nr_part_plan_info(int coords, const int Nxx[3], int NG, const int parts[3], int64_t* nparts, int64_t records[4])
{
    return nrk_guard("nr_part_plan_info", [&]() -> int {
        HostSetup H;
        PartPlan plan;
        int rc = plan_host(coords, Nxx, NG, parts, H, plan);
        if (rc) return rc;
        if (nparts) *nparts = plan.np;
        if (records) {
            records[0] = 0;
            for (const auto& v : plan.inner) records[0] += (int64_t)v.size();
            for (const PartMsg& m : plan.msg[0]) records[0] += (int64_t)m.sidx.size();
            for (int ph = 1; ph < 4; ph++) {
                records[ph] = 0;
                for (const PartMsg& m : plan.msg[ph]) records[ph] += (int64_t)m.sidx.size();
            }
        }
        return NR_OK;
    });
}

int nr_part_plan_boxes(int coords, const int Nxx[3], int NG, const int parts[3], int32_t* boxes)
{
    return nrk_guard("nr_part_plan_boxes", [&]() -> int {
        if (!boxes) return nrk_fail(NR_EINVAL, "boxes is NULL");
        HostSetup H;
        PartPlan plan;
        int rc = plan_host(coords, Nxx, NG, parts, H, plan);
        if (rc) return rc;
        for (int q = 0; q < plan.np; q++) {
            const PartBox& b = plan.box[q];
            int32_t* o = boxes + 15 * q;
            for (int d = 0; d < 3; d++) {
                o[d] = b.lo[d];
                o[3 + d] = b.hi[d];
                o[6 + d] = b.olo[d];
                o[9 + d] = b.ohi[d];
                o[12 + d] = b.org[d];
            }
        }
        return NR_OK;
    });
}

int nr_part_plan_records(int coords, const int Nxx[3], int NG, const int parts[3], int phase, int32_t* rec,
                         int64_t capacity)
{
    return nrk_guard("nr_part_plan_records", [&]() -> int {
        if (!rec || phase < 0 || phase > 3) return nrk_fail(NR_EINVAL, "bad nr_part_plan_records arguments");
        HostSetup H;
        PartPlan plan;
        int rc = plan_host(coords, Nxx, NG, parts, H, plan);
        if (rc) return rc;
        int64_t k = 0;
        auto put = [&](int sp, int sl, int dp, int dl, int neg) {
            if (k >= capacity) return false;
            int32_t* o = rec + 5 * k++;
            o[0] = sp;
            o[1] = sl;
            o[2] = dp;
            o[3] = dl;
            o[4] = neg;
            return true;
        };
        if (phase == 0)
            for (int q = 0; q < plan.np; q++)
                for (const InnerPt& p : plan.inner[q])
                    if (!put(q, p.src, q, p.dst, p.negmask)) return nrk_fail(NR_EINVAL, "capacity too small");
        for (const PartMsg& m : plan.msg[phase])
            for (size_t t = 0; t < m.sidx.size(); t++)
                if (!put(m.src, m.sidx[t], m.dst, m.didx[t], phase == 0 ? m.neg[t] : 0))
                    return nrk_fail(NR_EINVAL, "capacity too small");
        return NR_OK;
    });
}

}  // extern "C"
