// C ABI of the adjoint form: checkpoint store of the forward run, and the reverse sweep that
// recomputes one checkpoint interval at a time (replay with the stage record on) and runs the
// reverse kernel over it.  See include/cmx.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cmx_problem.h"

using namespace cmx;
using namespace cmx_host;

namespace cmx_host {

struct AdjState {
    int every = 0, slots = 0;
    long long max_steps = 0, base_log = 0;
    float *traj_m = nullptr, *traj_k = nullptr;
    double *traj_a = nullptr;
    // reverse sweep (allocated by the first cmx_adjoint)
    bool ready = false;
    float *rm[2] = {nullptr, nullptr}, *rk[7] = {};
    Ctl *rctl = nullptr;
    float *rec_m = nullptr;
    double *rec_a = nullptr, *rec_t = nullptr;
    double *dts = nullptr, *dl = nullptr;
    long long dts_cap = 0, dl_cap = 0;
    float *F[5] = {}, *mbar = nullptr, *k1bar = nullptr, *ubar = nullptr;
    double *ubar64 = nullptr;
    AdjCtl *actl = nullptr;
    int4 *tiles = nullptr;
    int *seg_begin = nullptr;
    int blocks = 0;
    float2 *part = nullptr;
};

void adj_free(cmx_problem *h)
{
    AdjState *s = h->adj;
    if (!s) return;
    void *ptrs[] = {s->traj_m, s->traj_k, s->traj_a, s->rm[0], s->rm[1], s->rctl, s->rec_m,
                    s->rec_a, s->rec_t, s->dts, s->dl, s->mbar, s->k1bar, s->ubar, s->ubar64, s->actl,
                    s->tiles, s->seg_begin, s->part};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (float *p : s->rk)
        if (p) cudaFree(p);
    for (float *p : s->F)
        if (p) cudaFree(p);
    delete s;
    h->adj = nullptr;
}

}  // namespace cmx_host

namespace {

// Start of a recompute interval: integrator state from checkpoint slot (a, k1^a), FSAL slope
// present, replay of n steps from dts.
__global__ void adj_restore_kernel(Ctl *ctl, const double *slot, int N, const double *dts,
                                   long long n)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int q = 0; q < 2 * N; q++) {
        ctl->a[q] = slot[q];
        ctl->ka[0][q] = slot[2 * N + q];
        ctl->mm_n[q] = slot[4 * N + q];
    }
    for (int j = 0; j < 7; j++) ctl->kphys[j] = j;
    ctl->t = slot[6 * N];   // the checkpoint's time (the drive depends on it)
    ctl->T = INFINITY;
    ctl->dt = dts[0];
    ctl->mcur = 0;
    ctl->k1_valid = 1;
    ctl->last_rejected = 0;
    ctl->status = 0;
    ctl->done = 0;
    ctl->replay = 1;
    ctl->replay_pos = 0;
    ctl->replay_n = n;
    ctl->replay_dts = dts;
    ctl->attempts = ctl->accepted = ctl->launch_attempts = 0;
    ctl->max_launch_attempts = n;
    ctl->rhs_evals = 0;
    ctl->log_n = ctl->trace_n = 0;
    ctl->trace_next = 0.0;
    ctl->bar_count = 0;
    ctl->skip_block = -1;
    for (int k = 0; k < 3; k++) {
        for (int q = 0; q < 2 * MAXN; q++) ctl->racc[k][q] = 0;
        ctl->remax[k] = 0u;
    }
    ctl->range_error = 0;
}

// FP64 running sum of the interval accumulators of dL/du, which are cleared.
__global__ void adj_fold_kernel(float *acc, double *total, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        total[i] += (double)acc[i];
        acc[i] = 0.f;
    }
}

__global__ void adj_scatter_d_kernel(const double *compact, double *dense, const int *box_of_cell,
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

int ensure_reverse(cmx_problem *h)
{
    AdjState *s = h->adj;
    if (s->ready) return CMX_OK;
    const int nq = 3 * h->grid.nsub, N = std::max(1, h->N);
    const size_t nc = (size_t)h->ncell;
    for (int b = 0; b < 2; b++) CU(dalloc(&s->rm[b], nq * nc));
    for (int j = 0; j < 7; j++) CU(dalloc(&s->rk[j], nq * nc));
    CU(cudaMemsetAsync(s->rm[1], 0, nq * nc * sizeof(float), h->stream));
    for (int j = 0; j < 7; j++) CU(cudaMemsetAsync(s->rk[j], 0, nq * nc * sizeof(float), h->stream));
    CU(dalloc(&s->rctl, 1));
    CU(dalloc(&s->rec_m, (size_t)s->every * 6 * nq * nc));
    CU(dalloc(&s->rec_a, (size_t)s->every * 7 * 4 * N));
    CU(dalloc(&s->rec_t, (size_t)s->every));
    for (int j = 0; j < 5; j++) CU(dalloc(&s->F[j], nq * nc));
    CU(dalloc(&s->mbar, nq * nc));
    CU(dalloc(&s->k1bar, nq * nc));
    if (h->u) {
        CU(dalloc(&s->ubar, (size_t)h->N * nc));
        CU(dalloc(&s->ubar64, (size_t)h->N * nc));
    }
    CU(dalloc(&s->actl, 1));
    // reverse partition: 32 x 8 windows, as many resident blocks as the kernel allows
    const int occ = reverse_blocks_per_sm(h->grid.nsub, h->u != nullptr);
    if (occ <= 0) return fail(h, CMX_ECUDA, "reverse kernel occupancy query failed");
    // (a window of REV_WX x REV_WY threads computes its interior, rim excluded)
    const std::vector<Column> cols = build_columns(h->lay, REV_WX - 2, REV_WY - 2);
    long long P = 0;
    for (const Column &c : cols) P += c.zhi - c.zlo;
    const int bz = std::max(1, h->bz);
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>((long long)occ * h->nsm, (P + bz - 1) / bz));
    std::vector<int4> segs;
    std::vector<int> begin;
    if (!build_segments(cols, blocks, segs, begin))
        return fail(h, CMX_EINVAL, "reverse partition: %zu columns do not fit %d blocks",
                    cols.size(), blocks);
    if (segs.empty()) return fail(h, CMX_EINVAL, "no tiles");
    CU(dalloc(&s->tiles, segs.size()));
    CU(dalloc(&s->seg_begin, begin.size()));
    CU(cudaMemcpy(s->tiles, segs.data(), segs.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(s->seg_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice));
    s->blocks = blocks;
    CU(dalloc(&s->part, (size_t)blocks * (N + 1)));
    s->ready = true;
    return CMX_OK;
}

// Accepted step sizes of the recorded run, from the step log.
int recorded_steps(cmx_problem *h, const Ctl &hc, std::vector<double> &dts)
{
    AdjState *s = h->adj;
    const long long n_log = hc.log_n - s->base_log;
    if (hc.log_n > h->sv.log_cap)
        return fail(h, CMX_EINVAL,
                    "the step log overflowed (%lld attempts, log_cap %d): the adjoint needs every "
                    "attempt of the run", hc.log_n, h->sv.log_cap);
    std::vector<cmx_step> log(std::max<long long>(n_log, 1));
    if (n_log > 0)
        CU(cudaMemcpy(log.data(), h->log + s->base_log, n_log * sizeof(cmx_step),
                      cudaMemcpyDeviceToHost));
    dts.clear();
    for (long long i = 0; i < n_log; i++)
        if (log[i].accepted) dts.push_back(log[i].dt);
    if ((long long)dts.size() > s->max_steps)
        return fail(h, CMX_EINVAL, "the run took %zu accepted steps, more than max_steps %lld",
                    dts.size(), s->max_steps);
    return CMX_OK;
}

}  // namespace

extern "C" {

int cmx_adjoint_record(cmx_problem *h, int every, long long max_steps)
{
    if (!h || every < 1 || max_steps < 1) return fail(h, CMX_EINVAL, "bad argument");
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    if (hc.k1_valid || hc.accepted != 0 || hc.attempts != 0)
        return fail(h, CMX_EINVAL, "cmx_adjoint_record must follow cmx_set_state directly");
    if (h->base.split_dt > 0.0)
        return fail(h, CMX_EINVAL, "the adjoint differentiates the coupled scheme, not the split one");
    if (h->base.fd)
        return fail(h, CMX_EINVAL, "the adjoint covers the diagonal demag factors only");
    if (!h->adj) h->adj = new AdjState();
    AdjState *s = h->adj;
    const int nq = 3 * h->grid.nsub, N = std::max(1, h->N);
    const size_t nc = (size_t)h->ncell;
    const long long slots = max_steps / every + 1;
    if (slots > (1LL << 30)) return fail(h, CMX_EINVAL, "max_steps / every too large");
    if (s->every != every || s->slots != slots) {
        // free what depends on the interval length or the slot count
        void *ptrs[] = {s->traj_m, s->traj_k, s->traj_a};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        s->traj_m = s->traj_k = nullptr;
        s->traj_a = nullptr;
        if (s->rec_m) cudaFree(s->rec_m);
        if (s->rec_a) cudaFree(s->rec_a);
        if (s->rec_t) cudaFree(s->rec_t);
        s->rec_m = nullptr;
        s->rec_a = nullptr;
        s->rec_t = nullptr;
        if (s->ready) {
            // the interval record is re-sized by ensure_reverse
            adj_free(h);
            h->adj = new AdjState();
            s = h->adj;
        }
        CU(dalloc(&s->traj_m, (size_t)slots * nq * nc));
        CU(dalloc(&s->traj_k, (size_t)slots * nq * nc));
        CU(dalloc(&s->traj_a, (size_t)slots * traj_stride(N)));
        s->every = every;
        s->slots = (int)slots;
    }
    s->max_steps = max_steps;
    s->base_log = hc.log_n;
    Ctx &c = h->base;
    c.traj_m = s->traj_m;
    c.traj_k = s->traj_k;
    c.traj_a = s->traj_a;
    c.traj_base = hc.accepted;
    c.traj_every = every;
    c.traj_slots = (int)slots;
    return CMX_OK;
}

int cmx_adjoint_steps(cmx_problem *h, long long *n)
{
    if (!h || !n) return fail(h, CMX_EINVAL, "bad argument");
    if (!h->adj || !h->base.traj_m) return fail(h, CMX_EINVAL, "nothing recorded");
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    *n = hc.accepted - h->base.traj_base;
    return CMX_OK;
}

int cmx_adjoint(cmx_problem *h, const double *dL_da, const float *dL_dm, int dL_dm_on_device,
                cmx_grads *g)
{
    if (!h || !g) return fail(h, CMX_EINVAL, "bad argument");
    if (!h->adj || !h->base.traj_m)
        return fail(h, CMX_EINVAL, "no run recorded: call cmx_adjoint_record before the run");
    AdjState *s = h->adj;
    Ctl hc;
    int rc = read_ctl(h, &hc);
    if (rc) return rc;
    if (hc.status) return device_status(h, hc);
    std::vector<double> dts;
    rc = recorded_steps(h, hc, dts);
    if (rc) return rc;
    const long long n = (long long)dts.size();
    if (n != hc.accepted - h->base.traj_base)
        return fail(h, CMX_EINVAL, "step log and accepted count disagree");
    const int N = h->N, nq = 3 * h->grid.nsub, Q = 2 * std::max(1, N);
    const size_t nc = (size_t)h->ncell;
    rc = ensure_reverse(h);
    if (rc) return rc;
    cudaStream_t st = h->stream;

    // inputs
    if (n + 1 > s->dl_cap) {
        if (s->dl) cudaFree(s->dl);
        s->dl = nullptr;
        s->dl_cap = 0;
        CU(dalloc(&s->dl, (size_t)(n + 1) * Q));
        s->dl_cap = n + 1;
    }
    if (std::max<long long>(n, 1) > s->dts_cap) {
        if (s->dts) cudaFree(s->dts);
        s->dts = nullptr;
        s->dts_cap = 0;
        CU(dalloc(&s->dts, std::max<long long>(n, 1)));
        s->dts_cap = std::max<long long>(n, 1);
    }
    if (n > 0) CU(cudaMemcpyAsync(s->dts, dts.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (dL_da && N > 0)
        CU(cudaMemcpyAsync(s->dl, dL_da, (size_t)(n + 1) * 2 * N * sizeof(double),
                           cudaMemcpyHostToDevice, st));
    // adjoint state at the end of the run
    CU(cudaMemsetAsync(s->mbar, 0, nq * nc * sizeof(float), st));
    if (dL_dm) {
        const float *src = dL_dm;
        if (!dL_dm_on_device) {
            CU(cudaMemcpyAsync(h->dense, dL_dm, (size_t)nq * h->nbox * sizeof(float),
                               cudaMemcpyHostToDevice, st));
            src = h->dense;
        }
        gather_kernel<<<grid_blocks((long long)nq * nc), 256, 0, st>>>(
            src, s->mbar, h->box_of_cell, h->active, h->ncell, h->nbox, nq);
        CU(cudaGetLastError());
    }
    CU(cudaMemsetAsync(s->k1bar, 0, nq * nc * sizeof(float), st));
    for (int j = 0; j < 5; j++) CU(cudaMemsetAsync(s->F[j], 0, nq * nc * sizeof(float), st));
    if (s->ubar) {
        CU(cudaMemsetAsync(s->ubar, 0, (size_t)N * nc * sizeof(float), st));
        CU(cudaMemsetAsync(s->ubar64, 0, (size_t)N * nc * sizeof(double), st));
    }
    AdjCtl a0;
    memset(&a0, 0, sizeof a0);
    for (int q = 0; q < 2 * N; q++) a0.abar[q] = dL_da ? dL_da[n * 2 * N + q] : 0.0;
    CU(cudaMemcpyAsync(s->actl, &a0, sizeof a0, cudaMemcpyHostToDevice, st));

    // recompute and reverse, last interval first
    const long long E = s->every;
    const long long nint = n > 0 ? (n + E - 1) / E : 0;
    Ctx fc = make_ctx(h);
    fc.m[0] = s->rm[0];
    fc.m[1] = s->rm[1];
    for (int j = 0; j < 7; j++) fc.k[j] = s->rk[j];
    fc.ctl = s->rctl;
    fc.log_cap = 0;
    fc.tr_cap = 0;
    fc.stage_only = 0;
    fc.traj_m = fc.traj_k = nullptr;
    fc.traj_a = nullptr;
    fc.rec_m = s->rec_m;
    fc.rec_a = s->rec_a;
    fc.rec_t = s->rec_t;
    AdjArgs A;
    memset(&A, 0, sizeof A);
    A.f = make_ctx(h);
    A.f.tiles = s->tiles;
    A.f.seg_begin = s->seg_begin;
    A.rec_m = s->rec_m;
    A.rec_a = s->rec_a;
    A.rec_t = s->rec_t;
    A.dL_da = (dL_da && N > 0) ? s->dl : nullptr;
    A.m_first = s->traj_m;
    A.a_first = s->traj_a;
    for (int j = 0; j < 5; j++) A.F[j] = s->F[j];
    A.mbar = s->mbar;
    A.k1bar = s->k1bar;
    A.ubar = s->ubar;
    A.ctl = s->actl;
    A.part = s->part;
    for (long long q = nint - 1; q >= 0; q--) {
        const long long first = q * E, len = std::min(E, n - first);
        CU(cudaMemcpyAsync(s->rm[0], s->traj_m + (size_t)q * nq * nc, nq * nc * sizeof(float),
                           cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(s->rk[0], s->traj_k + (size_t)q * nq * nc, nq * nc * sizeof(float),
                           cudaMemcpyDeviceToDevice, st));
        adj_restore_kernel<<<1, 32, 0, st>>>(s->rctl, s->traj_a + (size_t)q * traj_stride(N), N,
                                             s->dts + first, len);
        CU(cudaGetLastError());
        fc.rec_steps = (int)len;
        cudaError_t e = launch_single(fc, h->bx, h->by, h->blocks, st);
        if (e != cudaSuccess) return fail(h, CMX_ECUDA, "recompute launch: %s", cudaGetErrorString(e));
        CU(cudaMemsetAsync(&s->actl->bar_count, 0, sizeof(unsigned), st));
        A.dts = s->dts + first;
        A.step0 = first;
        A.nsteps = (int)len;
        e = launch_reverse(A, s->blocks, st);
        if (e != cudaSuccess) return fail(h, CMX_ECUDA, "reverse launch: %s", cudaGetErrorString(e));
        if (s->ubar) {
            adj_fold_kernel<<<grid_blocks((long long)N * nc), 256, 0, st>>>(s->ubar, s->ubar64,
                                                                           (long long)N * nc);
            CU(cudaGetLastError());
        }
        h->launches += 2;
    }

    // results
    AdjCtl ac;
    Ctl rcl;
    CU(cudaMemcpyAsync(&ac, s->actl, sizeof ac, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&rcl, s->rctl, sizeof rcl, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (nint > 0 && rcl.status) return device_status(h, rcl);
    if (ac.status == CMX_ETIMEOUT)
        return fail(h, CMX_ETIMEOUT, "reverse barrier wait exceeded %lld ns (stage %d)",
                    h->timeout_ns, ac.timeout_where);
    if (ac.status) return fail(h, ac.status, "reverse sweep status %d", ac.status);
    for (int k = 0; k < N; k++) {
        if (g->g_re) g->g_re[k] = ac.gacc[NGRAD * k + 0];
        if (g->g_im) g->g_im[k] = ac.gacc[NGRAD * k + 1];
        if (g->kappa) g->kappa[k] = ac.gacc[NGRAD * k + 2];
        if (g->omega) g->omega[k] = ac.gacc[NGRAD * k + 3];
        if (g->gb_re) g->gb_re[k] = ac.gacc[NGRAD * k + 4];
        if (g->gb_im) g->gb_im[k] = ac.gacc[NGRAD * k + 5];
        if (g->kerr) g->kerr[k] = ac.gacc[NGRAD * k + 6];
        if (g->pump_re) g->pump_re[k] = ac.gacc[NGRAD * k + 7];
        if (g->pump_im) g->pump_im[k] = ac.gacc[NGRAD * k + 8];
    }
    if (g->alpha) *g->alpha = ac.galpha;
    if (g->a0)
        for (int q = 0; q < 2 * N; q++) g->a0[q] = ac.abar[q];
    if (g->m0) {
        float *d = g->m0_on_device ? g->m0 : h->dense;
        CU(cudaMemsetAsync(d, 0, (size_t)nq * h->nbox * sizeof(float), st));
        scatter_kernel<<<grid_blocks((long long)nq * nc), 256, 0, st>>>(
            s->mbar, d, h->box_of_cell, h->active, h->ncell, h->nbox, nq);
        CU(cudaGetLastError());
        if (!g->m0_on_device)
            CU(cudaMemcpyAsync(g->m0, h->dense, (size_t)nq * h->nbox * sizeof(float),
                               cudaMemcpyDeviceToHost, st));
    }
    if (g->u) {
        if (!s->ubar64) return fail(h, CMX_EINVAL, "dL/du needs mode profiles");
        double *d = g->u;
        double *tmp = nullptr;
        if (!g->u_on_device) {
            CU(dalloc(&tmp, (size_t)N * h->nbox));
            d = tmp;
        }
        CU(cudaMemsetAsync(d, 0, (size_t)N * h->nbox * sizeof(double), st));
        adj_scatter_d_kernel<<<grid_blocks((long long)N * nc), 256, 0, st>>>(
            s->ubar64, d, h->box_of_cell, h->active, h->ncell, h->nbox, N);
        CU(cudaGetLastError());
        if (tmp) {
            cudaError_t e = cudaMemcpyAsync(g->u, tmp, (size_t)N * h->nbox * sizeof(double),
                                            cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            cudaFree(tmp);
            if (e != cudaSuccess) return fail(h, CMX_ECUDA, "dL/du copy: %s", cudaGetErrorString(e));
        }
    }
    CU(cudaStreamSynchronize(st));
    return CMX_OK;
}

}  // extern "C"
