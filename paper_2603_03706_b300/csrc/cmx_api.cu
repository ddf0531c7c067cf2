// C ABI of libcmx: problem set-up (compact layout and tiles), state transfer and the host loop
// around the persistent device integrator.  See include/cmx.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cmx_problem.h"

using namespace cmx;
using namespace cmx_host;

namespace cmx_host {

int fail(cmx_problem *h, int code, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

__global__ void gather_kernel(const float *dense, float *compact, const int *box_of_cell,
                              const uint32_t *active, int ncell, long long nbox, int nq)
{
    const long long total = (long long)nq * ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / ncell), c = (int)(i - (long long)q * ncell);
        const bool on = !active || ((active[c >> 5] >> (c & 31)) & 1u);
        compact[i] = on ? dense[q * nbox + box_of_cell[c]] : 0.f;
    }
}

__global__ void scatter_kernel(const float *compact, float *dense, const int *box_of_cell,
                               const uint32_t *active, int ncell, long long nbox, int nq)
{
    const long long total = (long long)nq * ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / ncell), c = (int)(i - (long long)q * ncell);
        const bool on = !active || ((active[c >> 5] >> (c & 31)) & 1u);
        if (on) dense[q * nbox + box_of_cell[c]] = compact[i];
    }
}

}  // namespace cmx_host

namespace {

// Normalise the magnetic cells of a freshly set state (inputs need not be exact unit vectors).
__global__ void normalise_kernel(float *m, const uint32_t *active, int ncell, int nsub)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const bool on = !active || ((active[c >> 5] >> (c & 31)) & 1u);
        for (int s = 0; s < nsub; s++) {
            float *x = m + (size_t)(3 * s) * ncell + c, *y = x + ncell, *z = y + ncell;
            if (!on) {
                *x = *y = *z = 0.f;
                continue;
            }
            const float n2 = *x * *x + *y * *y + *z * *z;
            const float r = n2 > 0.f ? rsqrtf(n2) : 0.f;
            *x *= r;
            *y *= r;
            *z *= r;
        }
    }
}

// Stream-ordered update of the run parameters in the control block before a launch.
__global__ void prep_kernel(Ctl *ctl, PrepArgs a)
{
    ctl->T = a.T;
    ctl->done = 0;
    ctl->launch_attempts = 0;
    ctl->max_launch_attempts = a.max_launch_attempts;
    ctl->skip_block = a.skip_block;
    ctl->bar_count = 0;
    if (a.set_replay == 1) {
        ctl->replay = 1;
        ctl->replay_pos = 0;
        ctl->replay_n = a.replay_n;
        ctl->replay_dts = a.replay_dts;
    } else if (a.set_replay == 0) {
        ctl->replay = 0;
    }
}

}  // namespace

int cmx_host::grid_blocks(long long n) { return (int)std::min<long long>(4096, (n + 255) / 256); }

namespace {

int install_tiling(cmx_problem *h, const std::vector<Column> &cols, int blocks, int bx, int by,
                   int bz, int occ);

int setup_tiling(cmx_problem *h, const cmx_tiling *t)
{
    int bx = 32, by = 8, bz = 0, bps = 0;
    h->bps_cap = t ? t->blocks_per_sm : 0;
    if (t && (t->bx || t->by)) {
        bx = t->bx;
        by = t->by;
    }
    if (t) {
        bz = t->bz;
        bps = t->blocks_per_sm;
    }
    if (!tile_shape_supported(h->grid.nsub, bx, by))
        return fail(h, CMX_EINVAL,
                    "tile %dx%d is not compiled for nsub=%d (32x4, 32x8, 32x16)", bx, by,
                    h->grid.nsub);
    // dense boxes take the tensor-copy stage path (not with the full-demag passes, which are
    // compiled into the per-thread-copy kernels)
    const bool dense = h->dense_ok && !h->plain_copies && !h->base.fd;
    int occ = single_blocks_per_sm(h->grid.nsub, bx, by, h->N > 0 && h->u != nullptr, dense);
    if (occ <= 0) return fail(h, CMX_ECUDA, "occupancy query failed for %dx%d", bx, by);
    if (bps > 0) occ = std::min(occ, bps);
    const std::vector<Column> cols = build_columns(h->lay, bx, by);
    long long P = 0;
    for (const Column &c : cols) P += c.zhi - c.zlo;
    // bz: the fewest planes a block should get (default 4); all resident blocks otherwise
    if (bz <= 0) bz = 4;
    const long long cap = (long long)occ * h->nsm;
    // with the full demag every resident block takes part in the FFT passes of each stage (their
    // lines are spread over the blocks), whatever the number of planes
    const int blocks = h->base.fd ? (int)std::max<long long>(1, cap)
                                  : (int)std::max<long long>(1, std::min<long long>(cap, (P + bz - 1) / bz));
    const int rc = install_tiling(h, cols, blocks, bx, by, bz, occ);
    if (rc == CMX_OK) h->base.dense = dense ? 1 : 0;
    return rc;
}

// Partition the columns among `blocks` blocks and upload the segments; record the shape.
int install_tiling(cmx_problem *h, const std::vector<Column> &cols, int blocks, int bx, int by,
                   int bz, int occ)
{
    std::vector<int4> segs;
    std::vector<int> begin;
    if (!build_segments(cols, blocks, segs, begin))
        return fail(h, CMX_EINVAL,
                    "%zu tile columns do not fit %d blocks of at most %d segments each "
                    "(use a larger tile)", cols.size(), blocks, MAX_BLOCK_SEGMENTS);
    if (segs.empty()) return fail(h, CMX_EINVAL, "no tiles");
    if (h->tiles) cudaFree(h->tiles);
    if (h->seg_begin) cudaFree(h->seg_begin);
    h->tiles = nullptr;
    h->seg_begin = nullptr;
    if (dalloc(&h->tiles, segs.size()) != cudaSuccess ||
        dalloc(&h->seg_begin, begin.size()) != cudaSuccess)
        return fail(h, CMX_ENOMEM, "tiles");
    cudaMemcpy(h->tiles, segs.data(), segs.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(h->seg_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice);
    h->ntiles = (int)segs.size();
    h->bx = bx;
    h->by = by;
    h->bz = bz;
    h->bps = occ;
    h->blocks = blocks;
    return CMX_OK;
}

// Single-block integrator: eligible when the magnetic cells' state, slopes, profiles and
// neighbour table fit one block's shared memory (at most SMALL_SMEM bytes); used unless the caller
// asked for a tile shape.  Builds the magnetic cells' stored indices and neighbour table.
constexpr size_t SMALL_SMEM = 200 * 1024;

int setup_small(cmx_problem *h, const cmx_tiling *t)
{
    const int nm = h->ncell_mag;
    const bool has_u = h->N > 0 && h->u != nullptr;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    const size_t need = small_smem_bytes(nm, h->grid.nsub, h->N, has_u);
    h->small_ok = need <= SMALL_SMEM && need + 8192 <= (size_t)optin;
    h->use_small = h->small_ok && !(t && (t->bx || t->by));
    h->small_default = h->use_small;
    if (!h->small_ok) return CMX_OK;
    const Layout &L = h->lay;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    std::vector<int> small_of_box((size_t)nx * ny * nz, -1), sidx(nm), snb(6 * (size_t)nm, -1);
    std::vector<int> box(nm);
    int k = 0;
    for (int i = 0; i < L.ncell; i++)
        if (L.active[i]) {
            sidx[k] = i;
            box[k] = L.box_of_cell[i];
            small_of_box[L.box_of_cell[i]] = k++;
        }
    for (int i = 0; i < nm; i++) {
        const int b = box[i], x = b % nx, y = (b / nx) % ny, z = b / (nx * ny);
        const int nbx[6] = {x > 0 ? b - 1 : -1, x + 1 < nx ? b + 1 : -1,
                            y > 0 ? b - nx : -1, y + 1 < ny ? b + nx : -1,
                            z > 0 ? b - nx * ny : -1, z + 1 < nz ? b + nx * ny : -1};
        for (int d = 0; d < 6; d++) snb[(size_t)d * nm + i] = nbx[d] >= 0 ? small_of_box[nbx[d]] : -1;
    }
    if (dalloc(&h->small_idx, nm) != cudaSuccess || dalloc(&h->small_nb, 6 * (size_t)nm) != cudaSuccess)
        return fail(h, CMX_ENOMEM, "small-grid tables");
    cudaMemcpy(h->small_idx, sidx.data(), nm * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(h->small_nb, snb.data(), snb.size() * sizeof(int), cudaMemcpyHostToDevice);
    return CMX_OK;
}

}  // namespace

int cmx_host::retile(cmx_problem *h, int bx, int by)
{
    const cmx_tiling t{bx, by, h->bz, h->bps_cap, h->plain_copies ? 1 : 0};
    return setup_tiling(h, &t);
}

Ctx cmx_host::make_ctx(const cmx_problem *h)
{
    Ctx c = h->base;
    c.tiles = h->tiles;
    c.seg_begin = h->seg_begin;
    c.ntiles = h->ntiles;
    c.bz = h->bz;
    c.timeout_ns = h->timeout_ns;
    return c;
}

namespace {

// The single-block integrator runs plain integrations of small grids; a run that records for
// the adjoint (checkpoints or stage values) takes the tiled kernel, which writes those stores.
bool small_run(const cmx_problem *h, const Ctx &c)
{
    return h->use_small && !c.traj_m && !c.rec_m && !c.stage_only;
}

int launch(cmx_problem *h, const PrepArgs &pa, const Ctx &c)
{
    prep_kernel<<<1, 1, 0, h->stream>>>(c.ctl, pa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, CMX_ECUDA, "prep launch: %s", cudaGetErrorString(e));
    e = small_run(h, c) ? launch_small(c, h->small_idx, h->small_nb, h->ncell_mag, h->stream)
                        : launch_single(c, h->bx, h->by, h->blocks, h->stream);
    if (e != cudaSuccess) return fail(h, CMX_ECUDA, "integrator launch: %s", cudaGetErrorString(e));
    h->launches++;
    return CMX_OK;
}

}  // namespace

int cmx_host::read_ctl(cmx_problem *h, Ctl *out)
{
    CU(cudaMemcpyAsync(out, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return CMX_OK;
}

namespace {

void fill_stats(const cmx_problem *h, const Ctl &c, cmx_stats *st)
{
    if (!st) return;
    st->t = c.t;
    st->dt = c.dt;
    st->attempts = c.attempts;
    st->accepted = c.accepted;
    st->cell_stage_updates = c.rhs_evals * (long long)h->ncell_mag;
    st->status = c.status;
    st->launches = h->launches;
}

}  // namespace

int cmx_host::device_status(cmx_problem *h, const Ctl &c)
{
    if (c.status == CMX_OK) return CMX_OK;
    if (c.status == CMX_ETIMEOUT)
        return fail(h, CMX_ETIMEOUT, "device barrier wait exceeded %lld ns (stage %d)",
                    h->timeout_ns, c.timeout_where);
    if (c.status == CMX_ENAN) return fail(h, CMX_ENAN, "error norm is NaN/Inf at t=%g", c.t);
    if (c.status == CMX_ESTEPFAIL)
        return fail(h, CMX_ESTEPFAIL, "step size below dt_min at t=%g", c.t);
    if (c.status == CMX_ECHECK)
        return fail(h, CMX_ECHECK, "device index check failed at site %d (index %lld)",
                    c.timeout_where, c.check_value);
    return fail(h, c.status, "device status %d", c.status);
}

namespace {

// Run launches until the integrator reports done because of T / replay end, an error, or the
// attempt budget.
int drive(cmx_problem *h, double T, long long max_attempts, int set_replay, long long replay_n,
          cmx_stats *st)
{
    Ctx c = make_ctx(h);
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    if (hc.status) return device_status(h, hc);
    const long long start = hc.attempts;
    bool first = true;
    for (;;) {
        long long budget = h->launch_attempts;
        if (max_attempts > 0) budget = std::min(budget, max_attempts - (hc.attempts - start));
        if (budget <= 0) break;
        if (set_replay != 1 && hc.t >= T) break;
        PrepArgs pa{};
        pa.T = T;
        pa.max_launch_attempts = budget;
        pa.set_replay = first ? set_replay : -1;
        pa.replay_n = replay_n;
        pa.replay_dts = h->replay_dts;
        pa.skip_block = first ? h->skip_block : -1;
        if (first) h->skip_block = -1;
        rc = launch(h, pa, c);
        if (rc) return rc;
        rc = read_ctl(h, &hc);
        if (rc) return rc;
        first = false;
        if (hc.status) {
            fill_stats(h, hc, st);
            return device_status(h, hc);
        }
        if (hc.replay && hc.replay_pos >= hc.replay_n) break;
        if (!hc.replay && hc.t >= T) break;
    }
    fill_stats(h, hc, st);
    return CMX_OK;
}

void free_all(cmx_problem *h)
{
    void *ptrs[] = {h->rows, h->active, h->box_of_cell, h->tiles, h->seg_begin, h->u,
                    h->mbuf[0], h->mbuf[1], h->msv[0], h->msv[1], h->esbuf, h->small_idx,
                    h->small_nb,
                    h->ctl, h->log, h->log_a, h->log_mm, h->tr_t, h->tr_a,
                    h->tr_mm, h->replay_dts, h->dense, h->ev_m, h->ev_k, h->ev_ctl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (float *p : h->kbuf)
        if (p) cudaFree(p);
    adj_free(h);
    demag_release(h);
}

int reset_ctl(cmx_problem *h, const double *a, double t)
{
    Ctl c;
    memset(&c, 0, sizeof c);
    c.t = t;
    c.T = t;
    c.dt = h->sv.dt0;
    for (int q = 0; q < 2 * h->N; q++) c.a[q] = a ? a[q] : 0.0;
    for (int j = 0; j < 7; j++) c.kphys[j] = j;
    c.trace_next = t;
    c.skip_block = -1;
    c.max_launch_attempts = 1;
    if (h->base.split_dt > 0.0) {   // operator-split scheme: a cavity step comes first
        c.split_t0 = t;
        c.split_next = t + h->base.split_dt;
        c.split_pending = 1;
    }
    CU(cudaMemcpyAsync(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return CMX_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
extern "C" {

const char *cmx_status_string(int s)
{
    switch (s) {
    case CMX_OK: return "ok";
    case CMX_EINVAL: return "invalid argument";
    case CMX_ENOMEM: return "out of memory";
    case CMX_ECUDA: return "CUDA error";
    case CMX_ENAN: return "NaN in error norm";
    case CMX_ESTEPFAIL: return "step size underflow";
    case CMX_ETIMEOUT: return "device wait timed out";
    case CMX_ESCRATCH: return "problem exceeds the fixed scratch of cmx_eval_rhs_noalloc";
    case CMX_ECHECK: return "device index check failed (bounds-checked build)";
    default: return "unknown status";
    }
}

const char *cmx_last_error(const cmx_problem *h) { return h ? h->err.c_str() : "null handle"; }

int cmx_checked_build(void) { return CMX_CHECK; }

int cmx_create(const cmx_grid *grid, const uint8_t *mask, const cmx_material *mat,
               const cmx_modes *modes, const cmx_solver *solver, const cmx_tiling *tiling,
               void *stream, cmx_problem **out)
{
    if (!out) return CMX_EINVAL;
    *out = nullptr;
    if (!grid || !mask || !mat || !solver) return CMX_EINVAL;
    if (grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0 || grid->nx > 65532 ||
        (grid->nsub != 1 && grid->nsub != 2) || !(grid->cx > 0) || !(grid->cy > 0) ||
        !(grid->cz > 0))
        return CMX_EINVAL;
    const int N = modes ? modes->n_modes : 0;
    if (N < 0 || N > MAXN) return CMX_EINVAL;
    if (N > 0 && (!modes->omega || !modes->kappa || !modes->g_re || !modes->g_im))
        return CMX_EINVAL;
    if (!(mat->Ms > 0) || !(mat->gamma > 0) || !(solver->rtol > 0) || !(solver->dt0 > 0) ||
        !(solver->dt_max > 0) || solver->log_cap < 0 || solver->trace_cap < 0)
        return CMX_EINVAL;
    const long long nbox = (long long)grid->nx * grid->ny * grid->nz;
    if (nbox > (1LL << 31) - 1) return CMX_EINVAL;

    cmx_problem *h = new (std::nothrow) cmx_problem();
    if (!h) return CMX_ENOMEM;
    h->grid = *grid;
    h->mat = *mat;
    h->sv = *solver;
    h->N = N;
    h->nbox = nbox;
    h->stream = (cudaStream_t)stream;
    for (int n = 0; n < N; n++) {
        h->omega[n] = modes->omega[n];
        h->kappa[n] = modes->kappa[n];
        h->gre[n] = modes->g_re[n];
        h->gim[n] = modes->g_im[n];
    }
    auto bail = [&](int rc) {
        free_all(h);
        delete h;
        return rc;
    };
    if (cudaGetDevice(&h->dev) != cudaSuccess) return bail(CMX_ECUDA);
    if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess)
        return bail(CMX_ECUDA);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev);
    if (!coop) return bail(CMX_ECUDA);

    // one cell per thread (the only kind of tile)
    const int tq = tiling ? tiling->plain_copies : 0;
    if (tq != 0 && tq != 1) return bail(CMX_EINVAL);
    h->plain_copies = tq == 1;
    build_layout(h->lay, grid->nx, grid->ny, grid->nz, mask);
    h->ncell = h->lay.ncell;
    h->ncell_mag = h->lay.ncell_mag;
    h->holes = h->lay.holes;
    {
        // dense storage: every (y, z) row magnetic over [0, nx), rows of nx rounded up to
        // ROW_ALIGN cells back to back
        bool full = !h->lay.holes;
        for (const int2 &r : h->lay.rows)
            full = full && (r.y & 0xffff) == 0 && (int)((unsigned)r.y >> 16) == grid->nx;
        const long long nxs = ((long long)grid->nx + ROW_ALIGN - 1) / ROW_ALIGN * ROW_ALIGN;
        h->dense_ok = full && (long long)h->ncell == nxs * grid->ny * grid->nz;
        h->base.nxs = (int)nxs;
    }
    if (h->ncell_mag == 0) return bail(CMX_EINVAL);
    const int nq = 3 * grid->nsub;
    const size_t nc = (size_t)h->ncell;
    // device buffers
    if (dalloc(&h->rows, h->lay.rows.size()) || dalloc(&h->box_of_cell, nc) ||
        dalloc(&h->mbuf[0], nq * nc) || dalloc(&h->mbuf[1], nq * nc) || dalloc(&h->ctl, 1) ||
        dalloc(&h->dense, (size_t)nq * nbox))
        return bail(CMX_ENOMEM);
    for (int j = 0; j < 7; j++)
        if (dalloc(&h->kbuf[j], nq * nc)) return bail(CMX_ENOMEM);
    if (dalloc(&h->msv[0], nq * nc) || dalloc(&h->msv[1], nq * nc) || dalloc(&h->esbuf, nq * nc))
        return bail(CMX_ENOMEM);
    cudaMemcpy(h->rows, h->lay.rows.data(), h->lay.rows.size() * sizeof(int2),
               cudaMemcpyHostToDevice);
    cudaMemcpy(h->box_of_cell, h->lay.box_of_cell.data(), nc * sizeof(int), cudaMemcpyHostToDevice);
    if (h->lay.padded) {   // gather / scatter skip inactive stored cells
        const std::vector<uint32_t> bits = active_bits(h->lay);
        if (dalloc(&h->active, bits.size())) return bail(CMX_ENOMEM);
        cudaMemcpy(h->active, bits.data(), bits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    }
    for (int j = 0; j < 7; j++) cudaMemset(h->kbuf[j], 0, nq * nc * sizeof(float));
    for (int j = 0; j < 2; j++) cudaMemset(h->msv[j], 0, nq * nc * sizeof(float));
    cudaMemset(h->esbuf, 0, nq * nc * sizeof(float));
    cudaMemset(h->mbuf[1], 0, nq * nc * sizeof(float));
    // mode profiles, compacted (umax bounds the overlap sums; device profiles: |u| <= 256)
    double umax = 1.0;
    if (N > 0 && modes->u) {
        if (dalloc(&h->u, (size_t)N * nc)) return bail(CMX_ENOMEM);
        if (modes->u_on_device) {
            umax = 256.0;
            gather_kernel<<<grid_blocks((long long)N * nc), 256>>>(
                modes->u, h->u, h->box_of_cell, h->active, h->ncell, nbox, N);
        } else {
            std::vector<float> uc((size_t)N * nc);
            for (int n = 0; n < N; n++)
                for (size_t i = 0; i < nc; i++) {
                    uc[n * nc + i] =
                        h->lay.active[i] ? modes->u[n * nbox + h->lay.box_of_cell[i]] : 0.f;
                    umax = std::max(umax, (double)std::fabs(uc[n * nc + i]));
                }
            cudaMemcpy(h->u, uc.data(), uc.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
    }
    // log and trace
    const int lc = std::max(1, solver->log_cap), tc = std::max(1, solver->trace_cap);
    const int Q = 2 * std::max(1, N);
    if (dalloc(&h->log, lc) || dalloc(&h->log_a, (size_t)lc * Q) ||
        dalloc(&h->log_mm, (size_t)lc * Q) || dalloc(&h->tr_t, tc) ||
        dalloc(&h->tr_a, (size_t)tc * Q) || dalloc(&h->tr_mm, (size_t)tc * Q))
        return bail(CMX_ENOMEM);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(CMX_ECUDA);

    // kernel context
    Ctx &c = h->base;
    memset(&c, 0, sizeof c);
    c.nx = grid->nx;
    c.ny = grid->ny;
    c.nz = grid->nz;
    c.nsub = grid->nsub;
    c.nmodes = N;
    c.ncell = h->ncell;
    c.ncell_mag = h->ncell_mag;
    c.nxs = (grid->nx + ROW_ALIGN - 1) / ROW_ALIGN * ROW_ALIGN;
    c.rows = h->rows;
    c.active = h->holes ? h->active : nullptr;   // the row spans exclude the padding
    c.u = h->u;
    c.m[0] = h->mbuf[0];
    c.m[1] = h->mbuf[1];
    for (int j = 0; j < 7; j++) c.k[j] = h->kbuf[j];
    c.msv[0] = h->msv[0];
    c.msv[1] = h->msv[1];
    c.es = h->esbuf;
    const double exch = 2.0 * mat->Aex / mat->Ms;
    c.wx = (float)(exch / (grid->cx * grid->cx));
    c.wy = (float)(exch / (grid->cy * grid->cy));
    c.wz = (float)(exch / (grid->cz * grid->cz));
    c.anis = (float)(2.0 * mat->Ku / mat->Ms);
    const double mu0 = 4.0e-7 * M_PI;
    for (int k = 0; k < 3; k++) {
        c.ku[k] = (float)mat->ku_axis[k];
        c.B0[k] = (float)mat->B0[k];
        c.dmg[k] = (float)(mu0 * mat->Ms * mat->Ndemag[k]);
    }
    c.BE = grid->nsub == 2 ? (float)mat->BE : 0.f;
    c.pre = (float)(-mat->gamma / (1.0 + mat->alpha * mat->alpha));
    c.alpha = (float)mat->alpha;
    for (int n = 0; n < N; n++) {
        c.omega[n] = h->omega[n];
        c.kappa[n] = h->kappa[n];
        c.gre[n] = h->gre[n];
        c.gim[n] = h->gim[n];
        c.gbre[n] = h->gre[n];   // reciprocal unless cmx_set_backward_coupling
        c.gbim[n] = h->gim[n];
    }
    c.two_over_gamma = 2.0 / mat->gamma;
    c.inv_nmag = 1.0 / (double)h->ncell_mag;
    c.red_scale = overlap_scale(umax * (double)h->ncell_mag);
    c.umax = (float)umax;
    c.rtol = solver->rtol;
    c.a_ref = solver->a_ref;
    c.dt_min = solver->dt_min;
    c.dt_max = solver->dt_max;
    c.sample_dt = solver->sample_dt;
    c.ctl = h->ctl;
    c.log = h->log;
    c.log_a = h->log_a;
    c.log_mm = h->log_mm;
    c.log_cap = solver->log_cap;
    c.tr_t = h->tr_t;
    c.tr_a = h->tr_a;
    c.tr_mm = h->tr_mm;
    c.tr_cap = solver->trace_cap;

    int rc = setup_tiling(h, tiling);
    if (rc) return bail(rc);
    rc = setup_small(h, tiling);
    if (rc) return bail(rc);

    // initial state: +z (sublattice 2: -z), a = 0
    std::vector<float> m0((size_t)nq * nc, 0.f);
    for (size_t i = 0; i < nc; i++)
        if (h->lay.active[i]) {
            m0[2 * nc + i] = 1.f;
            if (grid->nsub == 2) m0[5 * nc + i] = -1.f;
        }
    cudaMemcpy(h->mbuf[0], m0.data(), m0.size() * sizeof(float), cudaMemcpyHostToDevice);
    rc = reset_ctl(h, nullptr, 0.0);
    if (rc) return bail(rc);
    *out = h;
    return CMX_OK;
}

int cmx_destroy(cmx_problem *h)
{
    if (!h) return CMX_EINVAL;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return CMX_OK;
}

int cmx_set_state(cmx_problem *h, const float *m, int m_on_device, const double *a, double t)
{
    if (!h || !m) return fail(h, CMX_EINVAL, "null argument");
    const int nq = 3 * h->grid.nsub;
    const size_t nc = (size_t)h->ncell;
    if (m_on_device) {
        gather_kernel<<<grid_blocks((long long)nq * nc), 256, 0, h->stream>>>(
            m, h->mbuf[0], h->box_of_cell, h->active, h->ncell, h->nbox, nq);
    } else {
        CU(cudaMemcpyAsync(h->dense, m, (size_t)nq * h->nbox * sizeof(float),
                           cudaMemcpyHostToDevice, h->stream));
        gather_kernel<<<grid_blocks((long long)nq * nc), 256, 0, h->stream>>>(
            h->dense, h->mbuf[0], h->box_of_cell, h->active, h->ncell, h->nbox, nq);
    }
    normalise_kernel<<<grid_blocks((long long)nc), 256, 0, h->stream>>>(h->mbuf[0], h->active,
                                                                         h->ncell, h->grid.nsub);
    CU(cudaGetLastError());
    // a new state ends any checkpoint recording for the adjoint
    h->base.traj_m = h->base.traj_k = nullptr;
    h->base.traj_a = nullptr;
    return reset_ctl(h, a, t);
}

int cmx_run(cmx_problem *h, double T, long long max_attempts, cmx_stats *st)
{
    if (!h) return CMX_EINVAL;
    return drive(h, T, max_attempts, 0, 0, st);
}

int cmx_launch(cmx_problem *h, double T, int n_attempts)
{
    if (!h || n_attempts <= 0) return fail(h, CMX_EINVAL, "bad argument");
    PrepArgs pa{};
    pa.T = T;
    pa.max_launch_attempts = n_attempts;
    pa.set_replay = 0;
    pa.skip_block = -1;
    return launch(h, pa, make_ctx(h));
}

int cmx_replay(cmx_problem *h, const double *dts, long long n, cmx_stats *st)
{
    if (!h || (!dts && n > 0) || n < 0) return fail(h, CMX_EINVAL, "bad argument");
    if (n == 0) return cmx_sync(h, st);
    for (long long i = 0; i < n; i++)
        if (!(dts[i] > 0)) return fail(h, CMX_EINVAL, "replay step %lld is not positive", i);
    if (n > h->replay_cap) {
        if (h->replay_dts) cudaFree(h->replay_dts);
        h->replay_dts = nullptr;
        h->replay_cap = 0;
        CU(dalloc(&h->replay_dts, n));
        h->replay_cap = n;
    }
    CU(cudaMemcpyAsync(h->replay_dts, dts, n * sizeof(double), cudaMemcpyHostToDevice,
                       h->stream));
    return drive(h, INFINITY, 0, 1, n, st);
}

int cmx_sync(cmx_problem *h, cmx_stats *st)
{
    if (!h) return CMX_EINVAL;
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    fill_stats(h, hc, st);
    return device_status(h, hc);
}

int cmx_get_m(cmx_problem *h, float *dst, int on_device)
{
    if (!h || !dst) return fail(h, CMX_EINVAL, "null argument");
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    const int nq = 3 * h->grid.nsub;
    float *d = on_device ? dst : h->dense;
    CU(cudaMemsetAsync(d, 0, (size_t)nq * h->nbox * sizeof(float), h->stream));
    scatter_kernel<<<grid_blocks((long long)nq * h->ncell), 256, 0, h->stream>>>(
        h->mbuf[hc.mcur], d, h->box_of_cell, h->active, h->ncell, h->nbox, nq);
    CU(cudaGetLastError());
    if (!on_device)
        CU(cudaMemcpyAsync(dst, h->dense, (size_t)nq * h->nbox * sizeof(float),
                           cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return CMX_OK;
}

int cmx_get_a(cmx_problem *h, double *dst)
{
    if (!h || (!dst && h->N > 0)) return fail(h, CMX_EINVAL, "null argument");
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    for (int q = 0; q < 2 * h->N; q++) dst[q] = hc.a[q];
    return CMX_OK;
}

int cmx_get_log(cmx_problem *h, cmx_step *dst, double *a, double *mm, int cap, long long *n)
{
    if (!h || cap < 0) return fail(h, CMX_EINVAL, "bad argument");
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    if (n) *n = hc.log_n;
    const long long k = std::min<long long>({(long long)cap, hc.log_n, (long long)h->sv.log_cap});
    const int Q = 2 * h->N;
    if (k > 0) {
        if (dst) CU(cudaMemcpy(dst, h->log, k * sizeof(cmx_step), cudaMemcpyDeviceToHost));
        if (a && Q) CU(cudaMemcpy(a, h->log_a, k * Q * sizeof(double), cudaMemcpyDeviceToHost));
        if (mm && Q)
            CU(cudaMemcpy(mm, h->log_mm, k * Q * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return CMX_OK;
}

int cmx_get_trace(cmx_problem *h, double *t, double *a, double *mm, int cap, long long *n)
{
    if (!h || cap < 0) return fail(h, CMX_EINVAL, "bad argument");
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    if (n) *n = hc.trace_n;
    const long long k = std::min<long long>({(long long)cap, hc.trace_n, (long long)h->sv.trace_cap});
    const int Q = 2 * h->N;
    if (k > 0) {
        if (t) CU(cudaMemcpy(t, h->tr_t, k * sizeof(double), cudaMemcpyDeviceToHost));
        if (a && Q) CU(cudaMemcpy(a, h->tr_a, k * Q * sizeof(double), cudaMemcpyDeviceToHost));
        if (mm && Q) CU(cudaMemcpy(mm, h->tr_mm, k * Q * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return CMX_OK;
}

int cmx_eval_rhs(cmx_problem *h, const float *m, const double *a, float *dm, double *da,
                 double *mm)
{
    if (!h || !m || !dm) return fail(h, CMX_EINVAL, "null argument");
    const int nq = 3 * h->grid.nsub;
    const size_t nc = (size_t)h->ncell;
    if (!h->ev_m) {
        CU(dalloc(&h->ev_m, nq * nc));
        CU(dalloc(&h->ev_k, nq * nc));
        CU(dalloc(&h->ev_ctl, 1));
    }
    CU(cudaMemcpyAsync(h->dense, m, (size_t)nq * h->nbox * sizeof(float), cudaMemcpyHostToDevice,
                       h->stream));
    gather_kernel<<<grid_blocks((long long)nq * nc), 256, 0, h->stream>>>(
        h->dense, h->ev_m, h->box_of_cell, h->active, h->ncell, h->nbox, nq);
    Ctl c0;
    memset(&c0, 0, sizeof c0);
    for (int q = 0; q < 2 * h->N; q++) c0.a[q] = a ? a[q] : 0.0;
    for (int j = 0; j < 7; j++) c0.kphys[j] = j;
    c0.dt = h->sv.dt0;
    c0.T = 1.0;
    c0.skip_block = -1;
    c0.max_launch_attempts = 1;
    CU(cudaMemcpyAsync(h->ev_ctl, &c0, sizeof c0, cudaMemcpyHostToDevice, h->stream));
    Ctx c = make_ctx(h);
    c.m[0] = h->ev_m;
    c.m[1] = h->ev_m;
    for (int j = 0; j < 7; j++) c.k[j] = h->ev_k;
    c.ctl = h->ev_ctl;
    c.stage_only = 1;
    c.log_cap = 0;
    c.tr_cap = 0;
    c.traj_m = c.traj_k = nullptr;
    c.traj_a = nullptr;
    c.rec_m = nullptr;
    c.rec_a = nullptr;
    cudaError_t e = launch_single(c, h->bx, h->by, h->blocks, h->stream);
    if (e != cudaSuccess) return fail(h, CMX_ECUDA, "eval launch: %s", cudaGetErrorString(e));
    CU(cudaMemsetAsync(h->dense, 0, (size_t)nq * h->nbox * sizeof(float), h->stream));
    scatter_kernel<<<grid_blocks((long long)nq * nc), 256, 0, h->stream>>>(
        h->ev_k, h->dense, h->box_of_cell, h->active, h->ncell, h->nbox, nq);
    CU(cudaMemcpyAsync(dm, h->dense, (size_t)nq * h->nbox * sizeof(float), cudaMemcpyDeviceToHost,
                       h->stream));
    Ctl hc;
    CU(cudaMemcpyAsync(&hc, h->ev_ctl, sizeof hc, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (hc.status) return device_status(h, hc);
    for (int q = 0; q < 2 * h->N; q++) {
        if (da) da[q] = hc.ka[0][q];
        if (mm) mm[q] = hc.mm_n[q];
    }
    return CMX_OK;
}

// Checkpoint blob: a header (magic, version, the sizes that must match), the control block and
// the compact state m_n and FSAL slope k_1 of every stored cell.
namespace {
struct StateHeader {
    unsigned magic, version;
    int nx, ny, nz, nsub, nmodes, ncell, ncell_mag;
    unsigned ctl_bytes;
    long long nfloats;   // floats of m and of k1 each
};
constexpr unsigned STATE_MAGIC = 0x53584d43u;   // "CMXS"
constexpr unsigned STATE_VERSION = 1;

size_t state_bytes(const cmx_problem *h)
{
    return sizeof(StateHeader) + sizeof(Ctl) + 2 * (size_t)3 * h->grid.nsub * h->ncell * sizeof(float);
}
}  // namespace

int cmx_save_state(cmx_problem *h, void *blob, size_t cap, size_t *size)
{
    if (!h) return CMX_EINVAL;
    const size_t need = state_bytes(h);
    if (size) *size = need;
    if (!blob) return CMX_OK;   // size query
    if (cap < need) return fail(h, CMX_EINVAL, "state blob needs %zu bytes", need);
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    if (hc.status) return device_status(h, hc);
    unsigned char *b = static_cast<unsigned char *>(blob);
    StateHeader hd{STATE_MAGIC, STATE_VERSION, h->grid.nx, h->grid.ny, h->grid.nz, h->grid.nsub,
                   h->N, h->ncell, h->ncell_mag, (unsigned)sizeof(Ctl),
                   (long long)3 * h->grid.nsub * h->ncell};
    memcpy(b, &hd, sizeof hd);
    memcpy(b + sizeof hd, &hc, sizeof hc);
    float *m = reinterpret_cast<float *>(b + sizeof hd + sizeof hc);
    const size_t bytes = (size_t)hd.nfloats * sizeof(float);
    CU(cudaMemcpyAsync(m, h->mbuf[hc.mcur], bytes, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(m + hd.nfloats, h->kbuf[hc.kphys[0]], bytes, cudaMemcpyDeviceToHost,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return CMX_OK;
}

int cmx_load_state(cmx_problem *h, const void *blob, size_t size)
{
    if (!h || !blob) return fail(h, CMX_EINVAL, "null argument");
    if (size < sizeof(StateHeader)) return fail(h, CMX_EINVAL, "state blob too short");
    StateHeader hd;
    memcpy(&hd, blob, sizeof hd);
    if (hd.magic != STATE_MAGIC || hd.version != STATE_VERSION || hd.ctl_bytes != sizeof(Ctl))
        return fail(h, CMX_EINVAL, "not a state blob of this library version");
    if (hd.nx != h->grid.nx || hd.ny != h->grid.ny || hd.nz != h->grid.nz ||
        hd.nsub != h->grid.nsub || hd.nmodes != h->N || hd.ncell != h->ncell ||
        hd.ncell_mag != h->ncell_mag || size < state_bytes(h))
        return fail(h, CMX_EINVAL, "state blob is for another problem");
    const unsigned char *b = static_cast<const unsigned char *>(blob);
    Ctl hc;
    memcpy(&hc, b + sizeof hd, sizeof hc);
    // per-launch and device-side fields start afresh; a replay in progress is not resumed
    hc.done = 0;
    hc.launch_attempts = 0;
    hc.max_launch_attempts = 1;
    hc.replay = 0;
    hc.replay_dts = nullptr;
    hc.replay_pos = hc.replay_n = 0;
    hc.bar_count = hc.bar_gen = 0;
    memset(hc.racc, 0, sizeof hc.racc);
    memset(hc.remax, 0, sizeof hc.remax);
    hc.range_error = 0;
    hc.skip_block = -1;
    hc.timeout_where = 0;
    const float *m = reinterpret_cast<const float *>(b + sizeof hd + sizeof hc);
    const size_t bytes = (size_t)hd.nfloats * sizeof(float);
    CU(cudaMemcpyAsync(h->mbuf[hc.mcur], m, bytes, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->kbuf[hc.kphys[0]], m + hd.nfloats, bytes, cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaMemcpyAsync(h->ctl, &hc, sizeof hc, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    // a loaded state ends any checkpoint recording for the adjoint
    h->base.traj_m = h->base.traj_k = nullptr;
    h->base.traj_a = nullptr;
    return CMX_OK;
}

int cmx_ncells(const cmx_problem *h, long long *n_magnetic, long long *n_stored)
{
    if (!h) return CMX_EINVAL;
    if (n_magnetic) *n_magnetic = h->ncell_mag;
    if (n_stored) *n_stored = h->ncell;
    return CMX_OK;
}

int cmx_set_launch_attempts(cmx_problem *h, int n)
{
    if (!h || n <= 0) return fail(h, CMX_EINVAL, "bad argument");
    h->launch_attempts = n;
    return CMX_OK;
}

int cmx_set_timeout(cmx_problem *h, long long ns)
{
    if (!h || ns <= 0) return fail(h, CMX_EINVAL, "bad argument");
    h->timeout_ns = ns;
    return CMX_OK;
}

int cmx_debug_skip_arrival(cmx_problem *h, int block)
{
    if (!h || block >= h->blocks) return fail(h, CMX_EINVAL, "bad argument");
    h->skip_block = block;
    return CMX_OK;
}

int cmx_set_split(cmx_problem *h, double ds)
{
    if (!h || !(ds >= 0.0) || !std::isfinite(ds)) return fail(h, CMX_EINVAL, "bad argument");
    if (ds > 0.0 && h->base.traj_m)
        return fail(h, CMX_EINVAL, "the adjoint differentiates the coupled scheme, not the split one");
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    h->base.split_dt = ds;
    hc.split_t0 = hc.t;
    hc.split_k = 0;
    hc.split_next = hc.t + ds;
    hc.split_pending = ds > 0.0;
    hc.k1_valid = 0;   // the first slope follows the first cavity step
    CU(cudaMemcpyAsync(h->ctl, &hc, sizeof hc, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return CMX_OK;
}

int cmx_set_backward_coupling(cmx_problem *h, const double *gb_re, const double *gb_im)
{
    if (!h || (gb_re && !gb_im)) return fail(h, CMX_EINVAL, "bad argument");
    Ctx &c = h->base;
    for (int n = 0; n < h->N; n++) {
        c.gbre[n] = gb_re ? gb_re[n] : h->gre[n];
        c.gbim[n] = gb_re ? gb_im[n] : h->gim[n];
    }
    c.has_gb = gb_re != nullptr;
    return CMX_OK;
}

int cmx_set_kerr(cmx_problem *h, const double *kerr)
{
    if (!h) return CMX_EINVAL;
    for (int n = 0; n < MAXN; n++) h->base.kerr[n] = (kerr && n < h->N) ? kerr[n] : 0.0;
    return CMX_OK;
}

int cmx_set_pump(cmx_problem *h, const double *p_re, const double *p_im, const double *wp)
{
    if (!h) return CMX_EINVAL;
    Ctx &c = h->base;
    if (!p_re) {
        c.has_pump = 0;
        for (int n = 0; n < MAXN; n++) c.pump_re[n] = c.pump_im[n] = c.pump_w[n] = 0.0;
        return CMX_OK;
    }
    if (!p_im || !wp) return fail(h, CMX_EINVAL, "pump: p_im and wp are needed");
    for (int n = 0; n < h->N; n++)
        if (!std::isfinite(p_re[n]) || !std::isfinite(p_im[n]) || !std::isfinite(wp[n]))
            return fail(h, CMX_EINVAL, "pump: non-finite coefficient of mode %d", n);
    for (int n = 0; n < MAXN; n++) {
        c.pump_re[n] = n < h->N ? p_re[n] : 0.0;
        c.pump_im[n] = n < h->N ? p_im[n] : 0.0;
        c.pump_w[n] = n < h->N ? wp[n] : 0.0;
    }
    c.has_pump = 1;
    return CMX_OK;
}

int cmx_set_drive(cmx_problem *h, const double *eta_re, const double *eta_im, double t0,
                  double sigma)
{
    if (!h) return CMX_EINVAL;
    Ctx &c = h->base;
    if (!eta_re) {
        c.has_drive = 0;
        return CMX_OK;
    }
    if (!eta_im || !(sigma > 0) || !std::isfinite(t0))
        return fail(h, CMX_EINVAL, "drive: eta_im, sigma > 0 and a finite t0 are needed");
    for (int n = 0; n < MAXN; n++) {
        c.drive_re[n] = n < h->N ? eta_re[n] : 0.0;
        c.drive_im[n] = n < h->N ? eta_im[n] : 0.0;
    }
    c.drive_t0 = t0;
    c.drive_inv_sigma = 1.0 / sigma;
    c.has_drive = h->N > 0;
    return CMX_OK;
}

int cmx_autotune(cmx_problem *h, int attempts, cmx_tiling *chosen, double *us_per_attempt)
{
    if (!h || attempts <= 0) return fail(h, CMX_EINVAL, "bad argument");
    Ctl saved;
    int rc = read_ctl(h, &saved);
    if (rc) return rc;
    if (saved.status) return device_status(h, saved);
    const int nq = 3 * h->grid.nsub;
    const size_t bytes = (size_t)nq * h->ncell * sizeof(float);
    float *m_save = nullptr, *k_save = nullptr;
    CU(dalloc(&m_save, (size_t)nq * h->ncell));
    if (dalloc(&k_save, (size_t)nq * h->ncell) != cudaSuccess) {
        cudaFree(m_save);
        return fail(h, CMX_ENOMEM, "autotune scratch");
    }
    cudaStream_t st = h->stream;
    cudaMemcpyAsync(m_save, h->mbuf[saved.mcur], bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(k_save, h->kbuf[saved.kphys[0]], bytes, cudaMemcpyDeviceToDevice, st);
    auto restore = [&]() {
        cudaMemcpyAsync(h->mbuf[saved.mcur], m_save, bytes, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(h->kbuf[saved.kphys[0]], k_save, bytes, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(h->ctl, &saved, sizeof saved, cudaMemcpyHostToDevice, st);
        return cudaStreamSynchronize(st);
    };
    // candidates 0..2: the compiled tiles; 3: the single-block integrator (small grids only)
    constexpr int NC = 3, SB = NC;
    static const int cand[NC][2] = {{32, 4}, {32, 8}, {32, 16}};
    const int bz = h->bz, bps = h->bps_cap;
    double best = 1e300, tus[NC + 1];
    int bi = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int ci = 0; ci <= NC; ci++) {
        double us = NAN;
        const bool small = ci == SB;
        cmx_tiling t{small ? 0 : cand[ci][0], small ? 0 : cand[ci][1], bz, bps, h->plain_copies ? 1 : 0};
        h->use_small = small;
        // full demag runs on the 32 x 8 tiles only
        const bool allowed = !h->base.fd || (!small && t.bx == 32 && t.by == 8);
        if (!allowed ? false
            : small ? h->small_ok
                  : (tile_shape_supported(h->grid.nsub, t.bx, t.by) && setup_tiling(h, &t) == CMX_OK)) {
            PrepArgs pa{};
            pa.T = INFINITY;
            pa.set_replay = -1;
            pa.skip_block = -1;
            pa.max_launch_attempts = 1;
            int r1 = launch(h, pa, make_ctx(h));   // warm-up
            pa.max_launch_attempts = attempts;
            cudaEventRecord(e0, st);
            int r2 = r1 ? r1 : launch(h, pa, make_ctx(h));
            cudaEventRecord(e1, st);
            Ctl after;
            if (!r2 && read_ctl(h, &after) == CMX_OK && !after.status &&
                after.attempts > saved.attempts + 1) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                us = 1e3 * ms / (double)(after.attempts - saved.attempts - 1);
            }
        }
        tus[ci] = us;
        if (us_per_attempt) us_per_attempt[ci] = us;
        if (us == us && us < best) {
            best = us;
            bi = ci;
        }
        if (restore() != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(m_save);
    cudaFree(k_save);
    if (!(best < 1e300)) return fail(h, CMX_ECUDA, "autotune: no window could be timed");
    // the tiled partition stays installed in every case (the adjoint's recorded runs use it)
    int tb = bi == SB ? 1 : bi;
    if (bi == SB) {   // the single-block integrator won: keep the best tile for recorded runs
        double bt = 1e300;
        for (int ci = 0; ci < NC; ci++)
            if (tus[ci] == tus[ci] && tus[ci] < bt) {
                bt = tus[ci];
                tb = ci;
            }
    }
    cmx_tiling t{cand[tb][0], cand[tb][1], bz, bps, h->plain_copies ? 1 : 0};
    rc = setup_tiling(h, &t);
    if (rc) return rc;
    h->use_small = bi == SB;
    h->small_default = h->use_small;
    if (chosen) *chosen = bi == SB ? cmx_tiling{0, 0, bz, bps, h->plain_copies ? 1 : 0} : t;
    return CMX_OK;
}

int cmx_plan_tiling(const cmx_grid *grid, const uint8_t *mask, int bx, int by, int blocks,
                    long long *n_segments, long long *n_stored)
{
    if (!grid || !mask || blocks <= 0 || grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0 ||
        grid->nx > 65532 || (grid->nsub != 1 && grid->nsub != 2))
        return CMX_EINVAL;
    if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 31) - 1) return CMX_EINVAL;
    if (!tile_shape_supported(grid->nsub, bx, by)) return CMX_EINVAL;
    Layout lay;
    build_layout(lay, grid->nx, grid->ny, grid->nz, mask);
    if (n_stored) *n_stored = lay.ncell;
    if (lay.ncell_mag == 0) return CMX_EINVAL;
    std::vector<int4> segs;
    std::vector<int> begin;
    if (!build_segments(build_columns(lay, bx, by), blocks, segs, begin)) return CMX_EINVAL;
    if (n_segments) *n_segments = (long long)segs.size();
    return CMX_OK;
}

int cmx_get_tiling(const cmx_problem *h, int *bx, int *by, int *bz, int *blocks, int *tiles,
                   int *dense)
{
    if (!h) return CMX_EINVAL;
    if (dense) *dense = (!h->use_small && h->base.dense) ? 1 : 0;
    if (bx) *bx = h->use_small ? 0 : h->bx;
    if (by) *by = h->use_small ? 0 : h->by;
    if (bz) *bz = h->bz;
    if (blocks) *blocks = h->use_small ? 1 : h->blocks;
    if (tiles) *tiles = h->use_small ? 0 : h->ntiles;
    return CMX_OK;
}

}  // extern "C"
