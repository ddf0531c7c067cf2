// Persistent single-problem integrator: one team of all blocks of a cooperative launch.
#include "cmx_engine.cuh"
#include "cmx_kernels.h"

namespace cmx {

// Blocks of WX x WY threads (one cell each); registers held so that several blocks are resident
// per SM: four of 128 threads, two of 256, one of 512.
template <int NT>
struct MinBlocks {
    static constexpr int value = NT <= 128 ? 4 : (NT <= 256 ? 2 : 1);
};

template <int NS, int WX, int WY, bool HU>
__global__ void __launch_bounds__(WX *WY, (MinBlocks<WX * WY>::value)) run_kernel(Ctx c)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<StageSmem<NS, WX, WY, HU> *>(smem_raw);
    __shared__ Local L;
    __shared__ Coef cf;
    __shared__ int s_stop;
    const Team tm{(int)blockIdx.x, (int)gridDim.x, &c.ctl->bar_count};
    integrate(c, tm, sm, L, cf, s_stop);
}

// ---------------------------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------------------------
template <int NS, int WX, int WY, bool HU>
static cudaError_t launch_variant(const Ctx &c, int blocks, cudaStream_t s)
{
    auto *fn = run_kernel<NS, WX, WY, HU>;
    const size_t smem = sizeof(StageSmem<NS, WX, WY, HU>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    Ctx cc = c;
    void *args[] = {&cc};
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(blocks), dim3(WX * WY), args, smem,
                                       s);
}

template <int NS, int WX, int WY, bool HU>
static int occupancy_variant()
{
    auto *fn = run_kernel<NS, WX, WY, HU>;
    const size_t smem = sizeof(StageSmem<NS, WX, WY, HU>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, WX * WY, smem) != cudaSuccess)
        return 0;
    return nb;
}

// Compiled tiles (with and without mode profiles): 32 x 4, 32 x 8 and 32 x 16 cells for one
// and for two sublattices.
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
#define X(n, a, b)                                                                       \
    if (c.nsub == n && bx == a && by == b)                                               \
        return c.u ? launch_variant<n, a, b, true>(c, blocks, s)                         \
                   : launch_variant<n, a, b, false>(c, blocks, s);
    CMX_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

int single_blocks_per_sm(int nsub, int bx, int by, bool has_u)
{
#define X(n, a, b)                                                                       \
    if (nsub == n && bx == a && by == b)                                                 \
        return has_u ? occupancy_variant<n, a, b, true>() : occupancy_variant<n, a, b, false>();
    CMX_VARIANTS(X)
#undef X
    return 0;
}

}  // namespace cmx
