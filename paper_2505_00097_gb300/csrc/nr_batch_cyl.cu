// nr_batch_cyl.cu -- batched-mode kernels for cylindrical-like grids, 4th-order scheme.
#include "nr_batch_kernels.cuh"

namespace nrk {

NRK_BATCH_LAUNCH(cyl4, FAM_CYL, 1, 4)

}  // namespace nrk
