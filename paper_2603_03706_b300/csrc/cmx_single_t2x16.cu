// Tile 16 rows x 32 cells, 2 sublattice(s): instantiation of the single-problem kernel.
#include "cmx_single_kernel.cuh"

namespace cmx {
CMX_INSTANTIATE_TILES(2, 32, 16)
}  // namespace cmx
