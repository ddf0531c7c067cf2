// One-sublattice tiles of the batched integrator.
#include "cmx_batch_kernel.cuh"

namespace cmx {
CMX_INSTANTIATE_BATCH(1, 32, 4)
CMX_INSTANTIATE_BATCH(1, 32, 8)
CMX_INSTANTIATE_BATCH(1, 32, 16)
}  // namespace cmx
