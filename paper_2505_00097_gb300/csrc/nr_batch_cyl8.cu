// nr_batch_cyl8.cu -- batched-mode kernels for cylindrical-like grids, 8th-order scheme.
#include "nr_batch_kernels.cuh"

namespace nrk {

NRK_BATCH_LAUNCH(cyl8, FAM_CYL, 1, 8)

}  // namespace nrk
