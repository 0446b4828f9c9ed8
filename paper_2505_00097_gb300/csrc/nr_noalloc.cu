// nr_noalloc.cu -- Hamiltonian-constraint evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns every byte
// of device memory through its own pool or a fixed HBM budget, a caller that
// holds no nr_grid (creating one allocates four 24-gridfunction sets) and
// only wants to check a state it already has on the device, or a latency-
// critical loop that cannot afford cudaMalloc's implicit device
// synchronisation.  nr_hamiltonian_noalloc serves them: it is the
// Hamiltonian-constraint kernel of nr_hamiltonian with its scratch memory
// (per-axis reference-metric arrays, per-block partial norms, the reduced
// result) held in the file-scope device array below instead of grid-owned
// cudaMalloc buffers.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "bssn_point.cuh"
#include "nr_geo.cuh"
#include "nr_internal.h"

namespace nrk {

// Scratch layout (doubles): [0, 3*NA_MAXBLOCKS) per-block partials (sum H^2,
// max |H|, count), [NA_RESULT, NA_RESULT+3) the reduced norms, [NA_AXES, ..)
// the per-axis arrays of nr_internal.h.  512 KiB, held by every GPU that
// loads the library until the process exits.
constexpr int NA_DOUBLES = 65536;
constexpr int NA_MAXBLOCKS = 2048;
constexpr int NA_RESULT = 3 * NA_MAXBLOCKS;
constexpr int NA_AXES = NA_RESULT + 32;
constexpr int NA_AXES_MAX = NA_DOUBLES - NA_AXES;
constexpr int NA_MAXDEV = 64;
constexpr int NA_THREADS = 128;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

// per-axis arrays, same values as the host set-up of nr_grid_create (layout in nr_internal.h)
__global__ void k_na_axes(int coords, int fam, int n0, int n1, int n2, int NG, double dx0, double dx1, double dx2,
                          double lo0, double lo1, double lo2, double A0, double w0, double A2, double w2, double* ax0,
                          double* ax1, double* ax2)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n0) {
        const double x = lo0 + ((double)(t - NG) + 0.5) * dx0;
        double f0, f1, f2;
        if (coords == NR_SPHERICAL) {
            f0 = A0 * x;
            f1 = A0;
            f2 = 0.0;
        } else {
            const double s = sinh(1.0 / w0), sh = sinh(x / w0), ch = cosh(x / w0);
            f0 = A0 * sh / s;
            f1 = A0 * ch / (w0 * s);
            f2 = A0 * sh / (w0 * w0 * s);
        }
        ax0[t] = 1.0 / f1;
        ax0[n0 + t] = 1.0 / f0;
        ax0[2 * n0 + t] = f2 / (f1 * f1);
        ax0[3 * n0 + t] = f0;
    } else if (t < n0 + n1) {
        const int i = t - n0;
        const double x = lo1 + ((double)(i - NG) + 0.5) * dx1;
        if (fam == FAM_SPH) {
            ax1[i] = 1.0 / sin(x);
            ax1[n1 + i] = cos(x) / sin(x);
            ax1[2 * n1 + i] = sin(x);
            ax1[3 * n1 + i] = cos(x);
        } else {
            ax1[i] = sin(x);
            ax1[n1 + i] = cos(x);
        }
    } else if (t < n0 + n1 + n2) {
        const int i = t - n0 - n1;
        const double x = lo2 + ((double)(i - NG) + 0.5) * dx2;
        if (fam == FAM_SPH) {
            ax2[i] = sin(x);
            ax2[n2 + i] = cos(x);
        } else {
            const double s = sinh(1.0 / w2), sh = sinh(x / w2), ch = cosh(x / w2);
            const double f0 = A2 * sh / s, f1 = A2 * ch / (w2 * s), f2 = A2 * sh / (w2 * w2 * s);
            ax2[i] = 1.0 / f1;
            ax2[n2 + i] = f2 / (f1 * f1);
            ax2[2 * n2 + i] = f0;
        }
    }
}

// k_ham with a fixed number of blocks: each block strides over the interior
// points, so the partials fit the static scratch for any grid size
template <int FAM, int ORD>
__global__ void __launch_bounds__(NA_THREADS) k_na_ham(GridK G, const double* __restrict__ y, double* H, double rmin,
                                                        double rmax, double* partials)
{
    const long nint = (long)G.N0 * G.N1 * G.N2;
    double s2 = 0.0, mx = 0.0, cnt = 0.0;
    for (long t = (long)blockIdx.x * NA_THREADS + threadIdx.x; t < nint; t += (long)gridDim.x * NA_THREADS) {
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
            s2 += h * h;
            mx = fmax(mx, fabs(h));
            cnt += 1.0;
        }
    }
    __shared__ double sh[3][NA_THREADS];
    sh[0][threadIdx.x] = s2;
    sh[1][threadIdx.x] = mx;
    sh[2][threadIdx.x] = cnt;
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
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

namespace {
std::mutex g_na_mutex;
double* g_na_addr[NA_MAXDEV] = {nullptr};
}  // namespace

}  // namespace nrk

using namespace nrk;

extern "C" int nr_hamiltonian_noalloc(int coords, const int Nxx[3], const nr_params* params, const double* y_dev,
                                      double* H_dev, double* l2_out, double* linf_out)
{
    if (!params || !Nxx || !y_dev) return nrk_fail(NR_EINVAL, "nr_hamiltonian_noalloc: NULL argument");
    if (coords != NR_SINH_SPHERICAL && coords != NR_SINH_CYLINDRICAL && coords != NR_SPHERICAL)
        return nrk_fail(NR_EINVAL, "nr_hamiltonian_noalloc: unknown coordinate system");
    if (params->NG != 3 && params->NG != 5) return nrk_fail(NR_EINVAL, "nr_hamiltonian_noalloc: NG must be 3 or 5");
    const int NG = params->NG;
    int n[3];
    long T = 1;
    for (int d = 0; d < 3; d++) {
        if (Nxx[d] < 1 || Nxx[d] > (1 << 20)) return nrk_fail(NR_EINVAL, "nr_hamiltonian_noalloc: bad Nxx");
        n[d] = Nxx[d] + 2 * NG;
        T *= n[d];
    }
    if (T >= (1L << 31)) return nrk_fail(NR_EINVAL, "nr_hamiltonian_noalloc: grid too large");
    const int fam = coords == NR_SINH_CYLINDRICAL ? FAM_CYL : FAM_SPH;
    const long axes = fam == FAM_SPH ? 4L * n[0] + 4L * n[1] + 2L * n[2] : 4L * n[0] + 2L * n[1] + 3L * n[2];
    if (axes > NA_AXES_MAX)
        return nrk_fail(NR_EINVAL,
                        "nr_hamiltonian_noalloc: per-axis arrays need %ld doubles, the static scratch holds %d "
                        "(SinhSpherical/Spherical: 4 n0 + 4 n1 + 2 n2, SinhCylindrical: 4 n0 + 2 n1 + 3 n2, "
                        "n_d = N_d + 2 NG)",
                        axes, NA_AXES_MAX);
    const int dev = params->device;
    if (dev < 0 || dev >= NA_MAXDEV) return nrk_fail(NR_EINVAL, "nr_hamiltonian_noalloc: device out of range");
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return nrk_fail(NR_ECUDA, "nr_hamiltonian_noalloc: cudaGetDevice");
    if (cudaSetDevice(dev) != cudaSuccess) return nrk_fail(NR_ECUDA, "nr_hamiltonian_noalloc: cudaSetDevice");
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};

    // once per device, with the device current: the device address of the scratch array
    double* scratch;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return nrk_fail(NR_ECUDA, "nr_hamiltonian_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_na_addr[dev] = (double*)p;
        }
        scratch = g_na_addr[dev];
    }

    GridK K;
    memset(&K, 0, sizeof K);
    K.n0 = n[0];
    K.n1 = n[1];
    K.n2 = n[2];
    K.N0 = Nxx[0];
    K.N1 = Nxx[1];
    K.N2 = Nxx[2];
    K.NG = NG;
    K.fam = fam;
    K.ax = -1;
    K.ord = 2 * (NG - 1);
    K.T = T;
    double lo[3], hi[3], dx[3];
    if (fam == FAM_CYL) {
        lo[0] = 0.0; hi[0] = 1.0;
        lo[1] = -M_PI; hi[1] = M_PI;
        lo[2] = -1.0; hi[2] = 1.0;
    } else {
        lo[0] = 0.0; hi[0] = 1.0;
        lo[1] = 0.0; hi[1] = M_PI;
        lo[2] = -M_PI; hi[2] = M_PI;
    }
    for (int d = 0; d < 3; d++) {
        dx[d] = (hi[d] - lo[d]) / Nxx[d];
        K.inv_d1[d] = 1.0 / ((K.ord == 8 ? FD<8>::den1 : FD<4>::den1) * dx[d]);
        K.inv_d2[d] = 1.0 / ((K.ord == 8 ? FD<8>::den2 : FD<4>::den2) * dx[d] * dx[d]);
    }
    double* ax0 = scratch + NA_AXES;
    double* ax1 = ax0 + 4L * n[0];
    double* ax2 = ax1 + (fam == FAM_SPH ? 4L : 2L) * n[1];
    K.rfm.ax0 = ax0;
    K.rfm.ax1 = ax1;
    K.rfm.ax2 = ax2;

    cudaStream_t s = (cudaStream_t)params->stream;
    const int nax = n[0] + n[1] + n[2];
    k_na_axes<<<(nax + 127) / 128, 128, 0, s>>>(coords, fam, n[0], n[1], n[2], NG, dx[0], dx[1], dx[2], lo[0], lo[1],
                                                 lo[2], params->ampl[0], params->sinhw[0], params->ampl[2],
                                                 params->sinhw[2], ax0, ax1, ax2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && H_dev) e = cudaMemsetAsync(H_dev, 0, sizeof(double) * T, s);
    const long nint = (long)Nxx[0] * Nxx[1] * Nxx[2];
    const int nb = (int)std::min<long>(NA_MAXBLOCKS, (nint + NA_THREADS - 1) / NA_THREADS);
    if (e == cudaSuccess) {
        const double r0 = params->h_rmin, r1 = params->h_rmax;
        if (fam == FAM_SPH && NG == 5) k_na_ham<FAM_SPH, 8><<<nb, NA_THREADS, 0, s>>>(K, y_dev, H_dev, r0, r1, scratch);
        else if (fam == FAM_SPH) k_na_ham<FAM_SPH, 4><<<nb, NA_THREADS, 0, s>>>(K, y_dev, H_dev, r0, r1, scratch);
        else if (NG == 5) k_na_ham<FAM_CYL, 8><<<nb, NA_THREADS, 0, s>>>(K, y_dev, H_dev, r0, r1, scratch);
        else k_na_ham<FAM_CYL, 4><<<nb, NA_THREADS, 0, s>>>(K, y_dev, H_dev, r0, r1, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_ham_reduce(scratch, nb, scratch + NA_RESULT, s);
    if (e == cudaSuccess && (l2_out || linf_out)) {
        double r[3];
        e = cudaMemcpyAsync(r, scratch + NA_RESULT, sizeof r, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            if (l2_out) *l2_out = r[0];
            if (linf_out) *linf_out = r[1];
        }
    }
    if (e != cudaSuccess) return nrk_fail(NR_ECUDA, "nr_hamiltonian_noalloc: %s", cudaGetErrorString(e));
    return NR_OK;
}
