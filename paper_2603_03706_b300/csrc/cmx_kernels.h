// Host-side entry points of the device code (implemented in the .cu files of this directory).
#pragma once

#include "cmx_internal.cuh"

namespace cmx {

// persistent single-problem integrator (cmx_single.cu)
bool tile_shape_supported(int nsub, int bx, int by);
cudaError_t launch_single(const Ctx &c, int bx, int by, int blocks, cudaStream_t s);
int single_blocks_per_sm(int nsub, int bx, int by, bool has_u);

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
