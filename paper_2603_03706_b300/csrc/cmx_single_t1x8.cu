// Tile 8 rows x 32 cells, 1 sublattice(s): instantiation of the single-problem kernel.
#include "cmx_single_kernel.cuh"

namespace cmx {
CMX_INSTANTIATE_TILES(1, 32, 8)
}  // namespace cmx
