// Persistent single-problem integrator: one team of all blocks of a cooperative launch.  The
// kernels are instantiated per tile shape in cmx_single_t*.cu; this file dispatches.
#include "cmx_kernels.h"

namespace cmx {

template <int NS, int WX, int WY>
cudaError_t launch_tiles(const Ctx &c, int blocks, cudaStream_t s);
template <int NS, int WX, int WY>
int occupancy_tiles(bool has_u, bool dense);

// Compiled tiles: 32 x 4, 32 x 8 and 32 x 16 cells for one and for two sublattices.
#define CMX_VARIANTS(X) \
    X(1, 32, 4) X(1, 32, 8) X(1, 32, 16) X(2, 32, 4) X(2, 32, 8) X(2, 32, 16)

bool tile_shape_supported(int nsub, int bx, int by)
{
#define X(n, a, b) if (nsub == n && bx == a && by == b) return true;
    CMX_VARIANTS(X)
#undef X
    return false;
}

cudaError_t launch_single(const Ctx &c, int bx, int by, int blocks, cudaStream_t s)
{
#define X(n, a, b) if (c.nsub == n && bx == a && by == b) return launch_tiles<n, a, b>(c, blocks, s);
    CMX_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

int single_blocks_per_sm(int nsub, int bx, int by, bool has_u, bool dense)
{
#define X(n, a, b) if (nsub == n && bx == a && by == b) return occupancy_tiles<n, a, b>(has_u, dense);
    CMX_VARIANTS(X)
#undef X
    return 0;
}

}  // namespace cmx
