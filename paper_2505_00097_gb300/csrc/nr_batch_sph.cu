// nr_batch_sph.cu -- batched-mode kernels for spherical-like grids, 4th-order scheme.
#include "nr_batch_kernels.cuh"

namespace nrk {

NRK_BATCH_LAUNCH(sph4, FAM_SPH, 2, 4)

}  // namespace nrk
