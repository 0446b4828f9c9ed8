// nr_batch_sph8.cu -- batched-mode kernels for spherical-like grids, 8th-order scheme.
#include "nr_batch_kernels.cuh"

namespace nrk {

NRK_BATCH_LAUNCH(sph8, FAM_SPH, 2, 8)

}  // namespace nrk
