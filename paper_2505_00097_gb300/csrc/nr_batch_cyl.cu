// nr_batch_cyl.cu -- batched-mode persistent kernels for cylindrical-like grids.
#include "nr_batch_kernels.cuh"

namespace nrk {

cudaError_t batch_stage_launch_cyl(bool two_point, int tile, const BGrid* g, int n, int total, int* counter, int stage,
                                   int blocks, cudaStream_t s)
{
    return two_point ? dispatch_stage<FAM_CYL, 1>(tile, g, n, total, counter, stage, blocks, s)
                     : dispatch_stage<FAM_CYL, -1>(tile, g, n, total, counter, stage, blocks, s);
}

int batch_occupancy_cyl(bool two_point, int tile, int sms)
{
    return two_point ? dispatch_occupancy<FAM_CYL, 1>(tile, sms) : dispatch_occupancy<FAM_CYL, -1>(tile, sms);
}

}  // namespace nrk
