// Persistent single-problem integrator: one team of all blocks of a cooperative launch.
#include "cmx_engine.cuh"
#include "cmx_kernels.h"
#include "cmx_quad.cuh"

namespace cmx {

// One block covers a WX x WY window; 256-thread blocks are held to 128 registers so that two
// of them are resident per SM.
template <int NS, int NT>
struct MinBlocks {
    static constexpr int value = NT <= 256 ? 2 : 1;
};

template <int NS, int WX, int WY, bool HU>
__global__ void __launch_bounds__(WX *WY, (MinBlocks<NS, WX * WY>::value)) run_kernel(Ctx c)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<StageSmem<NS, WX, WY, HU> *>(smem_raw);
    __shared__ Local L;
    __shared__ Coef cf;
    __shared__ int s_stop;
    const Team tm{(int)blockIdx.x, (int)gridDim.x, &c.ctl->bar_count};
    integrate(c, tm, sm, L, cf, s_stop);
}

// Quad windows (one sublattice): wq x wy threads, four x-cells each; one block per SM.
template <bool HU>
__global__ void __launch_bounds__(QMAX_NT, 1) run_kernel_quad(Ctx c, int wq, int wy)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    QuadSmem<HU> sm = quad_smem<HU>(smem_raw, wq, wy, c.nmodes);
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

// Compiled block windows (with and without mode profiles): four for one sublattice, the
// 256-thread ones for two (larger two-sublattice windows would not leave room for two blocks).
#define CMX_VARIANTS(X) \
    X(1, 32, 8) X(1, 32, 16) X(1, 64, 4) X(2, 32, 8) X(2, 32, 16) X(2, 64, 4)

template <bool HU>
static cudaError_t launch_quad(const Ctx &c, int wq, int wy, int blocks, cudaStream_t s)
{
    auto *fn = run_kernel_quad<HU>;
    const size_t smem = quad_smem_bytes(wq * wy, HU ? c.nmodes : 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    Ctx cc = c;
    void *args[] = {&cc, &wq, &wy};
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(blocks), dim3(wq * wy), args, smem,
                                       s);
}

bool quad_shape_supported(int wq, int wy)
{
    return wq >= 3 && wy >= 3 && wy <= QMAX_WY && wq * wy <= QMAX_NT && (wq * wy) % 32 == 0;
}

int quad_blocks_per_sm(int wq, int wy, int nu)
{
    const int nt = wq * wy;
    const size_t smem = quad_smem_bytes(nt, nu);
    int nb = 0;
    if (nu > 0) {
        auto *fn = run_kernel_quad<true>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nt, smem) != cudaSuccess)
            return 0;
    } else {
        auto *fn = run_kernel_quad<false>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nt, smem) != cudaSuccess)
            return 0;
    }
    return nb;
}

bool tile_shape_supported(int nsub, int bx, int by)
{
#define X(n, a, b) if (nsub == n && bx == a && by == b) return true;
    CMX_VARIANTS(X)
#undef X
    return false;
}

cudaError_t launch_single(const Ctx &c, int bx, int by, int blocks, cudaStream_t s)
{
    if (c.quad) {
        if (c.nsub != 1 || bx % 4 || !quad_shape_supported(bx / 4, by)) return cudaErrorInvalidValue;
        return c.u ? launch_quad<true>(c, bx / 4, by, blocks, s)
                   : launch_quad<false>(c, bx / 4, by, blocks, s);
    }
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
