// Host-side state of one problem handle and the helpers shared by the C-ABI source files.
#pragma once

#include <string>

#include "cmx_kernels.h"
#include "cmx_layout.h"

namespace cmx_host {
struct AdjState;
}

using cmx::Ctl;
using cmx::Ctx;
using cmx::Layout;
using cmx::MAXN;

struct cmx_problem {
    int dev = 0;
    cudaStream_t stream = nullptr;
    cmx_grid grid{};
    cmx_material mat{};
    cmx_solver sv{};
    int N = 0;
    double omega[MAXN]{}, kappa[MAXN]{}, gre[MAXN]{}, gim[MAXN]{};
    long long nbox = 0;
    int ncell = 0, ncell_mag = 0;
    bool holes = false;   // holes inside a row's magnetic span (stage kernels test them)
    bool dense_ok = false;      // every row is magnetic over the whole box (dense storage)
    bool plain_copies = false;  // cmx_tiling.plain_copies: no tensor-copy stage path
    Layout lay;
    // device buffers
    int2 *rows = nullptr;
    uint32_t *active = nullptr;
    int *box_of_cell = nullptr;
    int4 *tiles = nullptr;
    int *seg_begin = nullptr;
    int ntiles = 0;
    float *u = nullptr;
    float *mbuf[2] = {nullptr, nullptr};
    float *kbuf[7] = {};
    float *msv[2] = {nullptr, nullptr};   // stored stage values
    float *esbuf = nullptr;               // error partial of stage 6
    Ctl *ctl = nullptr;
    cmx_step *log = nullptr;
    double *log_a = nullptr, *log_mm = nullptr;
    double *tr_t = nullptr, *tr_a = nullptr, *tr_mm = nullptr;
    double *replay_dts = nullptr;
    long long replay_cap = 0;
    float *dense = nullptr;           // nsub*3*nbox scratch for dense <-> compact
    // eval_rhs scratch
    float *ev_m = nullptr, *ev_k = nullptr;
    Ctl *ev_ctl = nullptr;
    // launch shape
    int bx = 32, by = 8, bz = 16, blocks = 0, bps = 0, nsm = 0;
    int bps_cap = 0;                  // blocks_per_sm requested (0 = as many as fit)
    // single-block integrator (small grids): magnetic cells' stored indices and neighbour table
    int *small_idx = nullptr, *small_nb = nullptr;
    bool small_ok = false;            // the grid fits one block's shared memory
    bool use_small = false;           // runs (not the adjoint's recorded ones) use it
    bool small_default = false;       // use_small as chosen at creation / by the autotuner
    // full demag (cmx_demag_api.cu)
    float *dm_k = nullptr;
    float2 *dm_work = nullptr, *dm_tw = nullptr;
    float *dm_bd = nullptr;
    long long launch_attempts = 4096;
    long long timeout_ns = 2000000000LL;
    int skip_block = -1;
    int launches = 0;
    std::string err;
    Ctx base{};
    cmx_host::AdjState *adj = nullptr;   // adjoint stores (cmx_adjoint_api.cu)
};


namespace cmx_host {

using namespace cmx;

// Record an error message on the handle and return the code.
int fail(cmx_problem *h, int code, const char *fmt, ...);

#define CU(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return cmx_host::fail(h, e_ == cudaErrorMemoryAllocation ? CMX_ENOMEM : CMX_ECUDA, \
                                  "%s failed: %s", #call, cudaGetErrorString(e_));         \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void **)p, n * sizeof(T));
}

int grid_blocks(long long n);
// dense box <-> compact cells, nq components
__global__ void gather_kernel(const float *dense, float *compact, const int *box_of_cell,
                              const uint32_t *active, int ncell, long long nbox, int nq);
__global__ void scatter_kernel(const float *compact, float *dense, const int *box_of_cell,
                               const uint32_t *active, int ncell, long long nbox, int nq);
Ctx make_ctx(const cmx_problem *h);
int read_ctl(cmx_problem *h, Ctl *out);
int device_status(cmx_problem *h, const Ctl &c);
void adj_free(cmx_problem *h);
void demag_release(cmx_problem *h);
// install the bx x by tile partition (bz and blocks_per_sm as before)
int retile(cmx_problem *h, int bx, int by);

}  // namespace cmx_host
