// Host-side entry points of the device code (implemented in the .cu files of this directory).
#pragma once

#include "cmx_internal.cuh"

namespace cmx {

// persistent single-problem integrator (cmx_single.cu)
bool tile_shape_supported(int nsub, int bx, int by);
cudaError_t launch_single(const Ctx &c, int bx, int by, int blocks, cudaStream_t s);
int single_blocks_per_sm(int nsub, int bx, int by, bool has_u);

// batched integrator (cmx_batch.cu)
struct BatchArgs {
    const Ctx *ctx;        // per instance
    const int *queue;      // instance indices; team t owns queue[q_begin[t] .. q_begin[t+1])
    const int *q_begin;
    int team_size;
};
cudaError_t launch_batch(const BatchArgs &b, int nsub, int bx, int by, int blocks, cudaStream_t s);
int batch_blocks_per_sm(int nsub, int bx, int by);
cudaError_t launch_batch_prep(Ctl *const *ctls, int n, long long max_attempts, cudaStream_t s);
cudaError_t launch_batch_pending(Ctl *const *ctls, int n, int *pending, cudaStream_t s);

// small helpers (cmx_api.cu)
struct PrepArgs {
    double T;
    long long max_launch_attempts;
    int set_replay;          // 1: switch to replay with the list below, 0: adaptive, -1: keep
    long long replay_n;
    const double *replay_dts;
    int skip_block;
};

}  // namespace cmx
