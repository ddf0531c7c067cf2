// Host-side entry points of the device code (implemented in the .cu files of this directory).
#pragma once

#include "cmx_internal.cuh"

namespace cmx {

// persistent single-problem integrator (cmx_single.cu); tiles of bx x by cells, one thread each
bool tile_shape_supported(int nsub, int bx, int by);
cudaError_t launch_single(const Ctx &c, int bx, int by, int blocks, cudaStream_t s);
int single_blocks_per_sm(int nsub, int bx, int by, bool has_u, bool dense = false);
// tensor maps of a dense launch (cmx_dense_maps.cu): the tile and operand boxes of its buffers
// for tiles of 32 x wy cells, in the order of the TM_* indices of cmx_dense.cuh; `map` points to
// `count` CUtensorMap objects (128 bytes each)
cudaError_t build_dense_maps(const Ctx &c, int wy, void *map, int count);

// single-block integrator for small grids (cmx_small.cu): sidx = stored index of each of the nm
// magnetic cells, snb = their neighbour table [-x, +x, -y, +y, -z, +z][nm] (-1: none)
size_t small_smem_bytes(int nm, int nsub, int nmodes, bool has_u);
cudaError_t launch_small(const Ctx &c, const int *sidx, const int *snb, int nm, cudaStream_t s);

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
// the external drive written into every instance's context (first nmodes amplitudes each)
struct DriveArgs {
    double re[MAXN], im[MAXN];
    double t0, inv_sigma;
    int on;
};
cudaError_t launch_batch_drive(Ctx *ctx, int n, const DriveArgs &d, cudaStream_t s);
// spectral map of the instances' uniform traces (one windowed DFT per instance)
struct SpecInst {
    const double *t, *a;     // trace times and packed amplitudes [k][q]
    const Ctl *ctl;          // trace_n
    int q, cap;              // amplitude stride (2 max(N, 1)), trace capacity
    int re;                  // column of Re a_mode, or -1 (the instance has no such mode)
};
cudaError_t launch_batch_spectrum(const SpecInst *si, int n, double f0, double df, int nf,
                                  double t_start, double *out, cudaStream_t s);

// reverse sweep of the adjoint (cmx_adjoint.cu)
// Scalar adjoint state in device memory, carried from one checkpoint interval to the previous.
constexpr int NGRAD = 9;   // scalar gradients per mode (see AdjCtl::gacc)

struct AdjCtl {
    double abar[2 * MAXN];           // dL/d a at the current step boundary
    double k1a[2 * MAXN];            // dL/d (cavity part of the FSAL slope)
    double gacc[NGRAD * MAXN];           // per mode: dL/d Re g~, Im g~, kappa, omega, Re gb~, Im gb~, K,
                                     // Re P, Im P (parametric pump)
    double galpha;                   // dL/d alpha
    unsigned int bar_count;          // arrival counter of the launch's barrier
    int status;
    int timeout_where;
};

struct AdjArgs {
    Ctx f;                           // problem (tiles / seg_begin: the reverse partition)
    const float *rec_m;              // stage points m_S, [j][S-2][nsub*3][ncell]
    const double *rec_a;             // a_S, <m^->_S, [j][S-1][2][2N]
    const double *rec_t;             // start time of step j of the interval (pump phase)
    const double *dts;               // step sizes of the interval
    const double *dL_da;             // [n+1][2N] by global state index, or NULL
    const float *m_first;            // initial state (stage-1 point of global step 0)
    const double *a_first;           // a_0, k1^a_0, <m^->(y_0): [3][2N]
    float *F[5];                     // adjoints of the stage points of stages 3..7
    float *mbar, *k1bar;             // dL/d m at the step boundary, dL/d (FSAL slope)
    float *ubar;                     // [N][ncell] interval accumulator of dL/d u, or NULL
    AdjCtl *ctl;
    float2 *part;                    // [blocks][N+1] block partials
    long long step0;                 // global index of the interval's first step
    int nsteps;
};
cudaError_t launch_reverse(const AdjArgs &a, int blocks, cudaStream_t s);
int reverse_blocks_per_sm(int nsub, bool has_u);
constexpr int REV_WX = 32, REV_WY = 8;   // window of the reverse kernel

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
