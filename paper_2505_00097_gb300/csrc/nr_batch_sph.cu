// nr_batch_sph.cu -- batched-mode kernels for spherical-like grids.
#include "nr_batch_kernels.cuh"

namespace nrk {

cudaError_t batch_stage_launch_sph(bool two_point, int tile, const BGrid* g, int n, int total, int stage,
                                   cudaStream_t s)
{
    return two_point ? dispatch_stage<FAM_SPH, 2>(tile, g, n, total, stage, s)
                     : dispatch_stage<FAM_SPH, -1>(tile, g, n, total, stage, s);
}

cudaError_t batch_d1_launch_sph(bool two_point, const BGrid* g, int n, int total_d1, int stage, cudaStream_t s)
{
    return two_point ? launch_batch_d1<2>(g, n, total_d1, stage, s) : launch_batch_d1<-1>(g, n, total_d1, stage, s);
}

}  // namespace nrk
