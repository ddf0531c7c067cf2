// Batched integrator kernel: one persistent cooperative launch advances many independent
// problems.  The blocks form teams of equal size; a team integrates the instances of its queue
// one after the other with the same engine as the single-problem kernel, synchronising only its
// own blocks through the instance's arrival counter.  Instantiated per tile shape in
// cmx_batch_t*.cu.
#pragma once

#include "cmx_engine.cuh"
#include "cmx_kernels.h"

namespace cmx {

template <int NS, int WX, int WY>
__global__ void __launch_bounds__(32 * WY, (WY <= 4 ? 4 : (WY <= 8 ? 2 : 1)))
    batch_kernel(BatchArgs B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<StageSmem<NS, WX, WY, false> *>(smem_raw);
    __shared__ Local L;
    __shared__ Coef cf;
    __shared__ int s_stop;
    __shared__ __align__(16) Ctx sc;
    const int team = blockIdx.x / B.team_size, rank = blockIdx.x % B.team_size;
    const int qb = __ldg(&B.q_begin[team]), qe = __ldg(&B.q_begin[team + 1]);
    for (int q = qb; q < qe; q++) {
        const int inst = __ldg(&B.queue[q]);
        // the instance's context into shared memory (word copy)
        const int *src = reinterpret_cast<const int *>(B.ctx + inst);
        int *dst = reinterpret_cast<int *>(&sc);
        for (int w = threadIdx.x; w < (int)(sizeof(Ctx) / sizeof(int)); w += 32 * WY)
            dst[w] = __ldg(src + w);
        __syncthreads();
        const Team tm{rank, B.team_size, &sc.ctl->bar_count};
        integrate<false>(sc, tm, sm, L, cf, s_stop);
    }
}

template <int NS, int WX, int WY>
static cudaError_t batch_launch_variant(const BatchArgs &b, int blocks, cudaStream_t s)
{
    auto *fn = batch_kernel<NS, WX, WY>;
    const size_t smem = sizeof(StageSmem<NS, WX, WY, false>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    BatchArgs bb = b;
    void *args[] = {&bb};
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(blocks), dim3(32 * WY), args, smem,
                                       s);
}

template <int NS, int WX, int WY>
static int batch_occupancy_variant()
{
    auto *fn = batch_kernel<NS, WX, WY>;
    const size_t smem = sizeof(StageSmem<NS, WX, WY, false>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * WY, smem) != cudaSuccess)
        return 0;
    return nb;
}

template <int NS, int WX, int WY>
cudaError_t batch_launch_tiles(const BatchArgs &b, int blocks, cudaStream_t s)
{
    return batch_launch_variant<NS, WX, WY>(b, blocks, s);
}

template <int NS, int WX, int WY>
int batch_occupancy_tiles()
{
    return batch_occupancy_variant<NS, WX, WY>();
}

#define CMX_INSTANTIATE_BATCH(NS, WX, WY)                                                       \
    template cudaError_t batch_launch_tiles<NS, WX, WY>(const BatchArgs &, int, cudaStream_t); \
    template int batch_occupancy_tiles<NS, WX, WY>();

}  // namespace cmx
