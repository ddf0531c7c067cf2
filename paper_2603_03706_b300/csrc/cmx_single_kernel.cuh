// Persistent single-problem integrator kernel and its launch helpers, instantiated per tile
// shape in the cmx_single_t*.cu files (one compilation unit each, so they build in parallel).
#pragma once

#include "cmx_dense.cuh"
#include "cmx_engine.cuh"
#include "cmx_kernels.h"

namespace cmx {

// Blocks of 32 x WY threads computing 32 x WY tiles (one cell per thread); registers held so
// that several blocks are resident per SM: four of 128 threads, two of 256, one of 512.
template <int NT>
struct MinBlocks {
    static constexpr int value = NT <= 128 ? 4 : (NT <= 256 ? 2 : 1);
};

// FD: compiled with the full-demag passes (only the 32 x 8 tiles; the plain kernels stay
// free of that code)
template <int NS, int WX, int WY, bool HU, bool FD>
__global__ void __launch_bounds__(32 * WY, (MinBlocks<32 * WY>::value)) run_kernel(Ctx c)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<StageSmem<NS, WX, WY, HU> *>(smem_raw);
    __shared__ Local L;
    __shared__ Coef cf;
    __shared__ int s_stop;
    const Team tm{(int)blockIdx.x, (int)gridDim.x, &c.ctl->bar_count};
    integrate<FD>(c, tm, sm, L, cf, s_stop);
}

// Dense-box kernel: the same engine with the tensor-copy stage path (cmx_dense.cuh).  Its
// tensor maps, built on the host from the launch's own buffers, arrive as a kernel parameter;
// the shared-memory struct starts on 128 bytes (the tensor copies' destinations).
template <int NS, int WY, bool HU>
__global__ void __launch_bounds__(32 * WY, (MinBlocks<32 * WY>::value))
    run_kernel_dense(const __grid_constant__ Ctx c, const __grid_constant__ DenseMaps maps)
{
    extern __shared__ __align__(16) unsigned char smem_dense[];
    unsigned char *base = smem_dense + ((128u - (smem_u32(smem_dense) & 127u)) & 127u);
    auto &sm = *reinterpret_cast<DenseSmem<NS, WY, HU> *>(base);
    __shared__ Local L;
    __shared__ Coef cf;
    __shared__ int s_stop;
    if (threadIdx.x == 0) sm.maps = &maps;
    const Team tm{(int)blockIdx.x, (int)gridDim.x, &c.ctl->bar_count};
    integrate<false>(c, tm, sm, L, cf, s_stop);
}

template <int NS, int WY, bool HU>
static size_t dense_smem_bytes()
{
    return sizeof(DenseSmem<NS, WY, HU>) + 128;
}

template <int NS, int WY, bool HU>
static cudaError_t launch_dense_variant(const Ctx &c, int blocks, cudaStream_t s)
{
    auto *fn = run_kernel_dense<NS, WY, HU>;
    const size_t smem = dense_smem_bytes<NS, WY, HU>();
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    DenseMaps maps;
    e = build_dense_maps(c, WY, maps.map, TM_COUNT);
    if (e != cudaSuccess) return e;
    Ctx cc = c;
    void *args[] = {&cc, &maps};
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(blocks), dim3(32 * WY), args, smem,
                                       s);
}

template <int NS, int WY, bool HU>
static int occupancy_dense_variant()
{
    auto *fn = run_kernel_dense<NS, WY, HU>;
    const size_t smem = dense_smem_bytes<NS, WY, HU>();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * WY, smem) != cudaSuccess)
        return 0;
    return nb;
}

template <int NS, int WX, int WY, bool HU, bool FD>
static cudaError_t launch_variant(const Ctx &c, int blocks, cudaStream_t s)
{
    auto *fn = run_kernel<NS, WX, WY, HU, FD>;
    const size_t smem = sizeof(StageSmem<NS, WX, WY, HU>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    Ctx cc = c;
    void *args[] = {&cc};
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(blocks), dim3(32 * WY), args, smem,
                                       s);
}

template <int NS, int WX, int WY, bool HU>
static int occupancy_variant()
{
    auto *fn = run_kernel<NS, WX, WY, HU, false>;
    const size_t smem = sizeof(StageSmem<NS, WX, WY, HU>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * WY, smem) != cudaSuccess)
        return 0;
    return nb;
}

template <int NS, int WX, int WY>
cudaError_t launch_tiles(const Ctx &c, int blocks, cudaStream_t s)
{
    if (c.dense && !c.fd)
        return c.u ? launch_dense_variant<NS, WY, true>(c, blocks, s)
                   : launch_dense_variant<NS, WY, false>(c, blocks, s);
    if (c.fd) {
        if constexpr (WX == 32 && WY == 8)
            return c.u ? launch_variant<NS, WX, WY, true, true>(c, blocks, s)
                       : launch_variant<NS, WX, WY, false, true>(c, blocks, s);
        return cudaErrorInvalidValue;   // full demag runs on the 32 x 8 tiles
    }
    return c.u ? launch_variant<NS, WX, WY, true, false>(c, blocks, s)
               : launch_variant<NS, WX, WY, false, false>(c, blocks, s);
}

template <int NS, int WX, int WY>
int occupancy_tiles(bool has_u, bool dense)
{
    if (dense)
        return has_u ? occupancy_dense_variant<NS, WY, true>()
                     : occupancy_dense_variant<NS, WY, false>();
    return has_u ? occupancy_variant<NS, WX, WY, true>() : occupancy_variant<NS, WX, WY, false>();
}

#define CMX_INSTANTIATE_TILES(NS, WX, WY)                                                    \
    template cudaError_t launch_tiles<NS, WX, WY>(const Ctx &, int, cudaStream_t);          \
    template int occupancy_tiles<NS, WX, WY>(bool, bool);

}  // namespace cmx
