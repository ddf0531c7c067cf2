// Two-sublattice tiles of the batched integrator.
#include "cmx_batch_kernel.cuh"

namespace cmx {
CMX_INSTANTIATE_BATCH(2, 32, 4)
CMX_INSTANTIATE_BATCH(2, 32, 8)
}  // namespace cmx
