// C ABI of the batched integrator (include/cmx.h, "Batched form"): per-instance layouts in
// shared device pools, team queues balanced by cell count, and the launch loop (optionally a
// captured CUDA graph) around the persistent batch kernel.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "cmx_kernels.h"
#include "cmx_layout.h"

using namespace cmx;

namespace {

struct Inst {
    cmx_grid grid{};
    cmx_material mat{};
    int N = 0;
    double omega[MAXN]{}, kappa[MAXN]{}, gre[MAXN]{}, gim[MAXN]{};
    double T = 0.0;
    Layout lay;
    std::vector<int4> segs;
    std::vector<int> begin;
    // offsets into the device pools
    size_t o_m[2] = {0, 0}, o_k[7] = {}, o_msv[2] = {0, 0}, o_es = 0, o_rows = 0, o_box = 0,
           o_act = 0, o_seg = 0, o_begin = 0, o_log = 0, o_loga = 0, o_tr = 0, o_tra = 0;
    bool has_act = false;        // active bitmask stored (padding or holes)
};

size_t up64(size_t n) { return (n + 63) & ~(size_t)63; }

}  // namespace

struct cmx_batch {
    int n = 0, nsub = 1, nsm = 0, dev = 0;
    int bx = 32, by = 8, team = 1, teams = 0, blocks = 0;
    cudaStream_t stream = nullptr;
    cmx_solver sv{};
    cmx_batch_config cfg{};
    std::vector<Inst> inst;
    long long cells = 0;
    // device pools
    float *fpool = nullptr;
    int2 *rows = nullptr;
    int *ipool = nullptr;        // box_of_cell and segment begins
    uint32_t *act = nullptr;
    int4 *segs = nullptr;
    Ctl *ctls = nullptr;
    Ctl **ctlp = nullptr;
    cmx_step *log = nullptr;
    double *logd = nullptr;      // log_a, log_mm
    double *trd = nullptr;       // tr_t, tr_a, tr_mm
    Ctx *ctx = nullptr;
    int *queue = nullptr, *qbegin = nullptr;
    int *pending = nullptr;
    int *pending_h = nullptr;
    float *dense = nullptr;
    size_t dense_cap = 0;
    // graph
    cudaGraphExec_t gexec = nullptr;
    int graph_attempts = 0;
    int graph_ok = 0;
    long long launches = 0;
    std::string err;
};

namespace {

int bfail(cmx_batch *b, int code, const char *fmt, ...)
{
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        b->err = buf;
    }
    return code;
}

#define BCU(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? CMX_ENOMEM : CMX_ECUDA,      \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

template <class T>
cudaError_t balloc(T **p, size_t n)
{
    *p = nullptr;
    return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
}

__global__ void bscatter_kernel(const float *compact, float *dense, const int *box_of_cell,
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

void free_batch(cmx_batch *b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    void *p[] = {b->fpool, b->rows, b->ipool, b->act, b->segs, b->ctls, b->ctlp,
                 b->log, b->logd, b->trd, b->ctx, b->queue, b->qbegin, b->pending,
                 b->dense};
    for (void *q : p)
        if (q) cudaFree(q);
    if (b->pending_h) cudaFreeHost(b->pending_h);
}

int enqueue_launch(cmx_batch *b, int attempts)
{
    cudaError_t e = launch_batch_prep(b->ctlp, b->n, attempts, b->stream);
    if (e == cudaSuccess) {
        BatchArgs a{b->ctx, b->queue, b->qbegin, b->team};
        e = launch_batch(a, b->nsub, b->bx, b->by, b->blocks, b->stream);
    }
    if (e == cudaSuccess) e = launch_batch_pending(b->ctlp, b->n, b->pending, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->pending_h, b->pending, sizeof(int), cudaMemcpyDeviceToHost,
                            b->stream);
    if (e != cudaSuccess) return bfail(b, CMX_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    return CMX_OK;
}

// One launch of `attempts` attempts per instance, from a captured graph when possible.
int run_once(cmx_batch *b, int attempts)
{
    if (b->cfg.use_graph) {
        if (b->gexec && b->graph_attempts != attempts) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        if (!b->gexec) {
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) ==
                      cudaSuccess;
            if (ok) ok = enqueue_launch(b, attempts) == CMX_OK;
            const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
            ok = ok && ec == cudaSuccess && g;
            if (ok) ok = cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();   // a refused capture leaves no error behind
            if (!ok) {
                b->gexec = nullptr;
                b->cfg.use_graph = 0;   // fall back to direct launches
                b->err.clear();
            } else {
                b->graph_attempts = attempts;
                b->graph_ok = 1;
            }
        }
        if (b->gexec) {
            BCU(cudaGraphLaunch(b->gexec, b->stream));
            b->launches++;
            return CMX_OK;
        }
    }
    const int rc = enqueue_launch(b, attempts);
    if (rc == CMX_OK) b->launches++;
    return rc;
}

int read_ctl(cmx_batch *b, int i, Ctl *out)
{
    BCU(cudaMemcpyAsync(out, b->ctls + i, sizeof(Ctl), cudaMemcpyDeviceToHost, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    return CMX_OK;
}

}  // namespace

extern "C" {

const char *cmx_batch_last_error(const cmx_batch *b) { return b ? b->err.c_str() : "null handle"; }

int cmx_batch_create(const cmx_instance *in, int n, const cmx_solver *solver,
                     const cmx_batch_config *cfg, void *stream, cmx_batch **out)
{
    if (!out) return CMX_EINVAL;
    *out = nullptr;
    if (!in || n <= 0 || !solver || !(solver->rtol > 0) || !(solver->dt0 > 0) ||
        solver->log_cap < 0 || solver->trace_cap < 0)
        return CMX_EINVAL;
    const int nsub = in[0].grid.nsub;
    for (int i = 0; i < n; i++) {
        const cmx_instance &d = in[i];
        const int N = d.modes.n_modes;
        if (!d.mask || d.grid.nsub != nsub || (nsub != 1 && nsub != 2) || d.grid.nx <= 0 ||
            d.grid.ny <= 0 || d.grid.nz <= 0 || d.grid.nx > 65535 || N < 0 || N > MAXN ||
            d.modes.u || !(d.mat.Ms > 0) || !(d.mat.gamma > 0) || !(d.T >= 0) ||
            (N > 0 && (!d.modes.omega || !d.modes.kappa || !d.modes.g_re || !d.modes.g_im)))
            return CMX_EINVAL;
    }
    cmx_batch *b = new (std::nothrow) cmx_batch();
    if (!b) return CMX_ENOMEM;
    auto bail = [&](int rc) {
        free_batch(b);
        delete b;
        return rc;
    };
    b->n = n;
    b->nsub = nsub;
    b->sv = *solver;
    b->stream = (cudaStream_t)stream;
    if (cfg) b->cfg = *cfg;
    else b->cfg.use_graph = 1;
    b->bx = b->cfg.bx ? b->cfg.bx : 32;
    b->by = b->cfg.by ? b->cfg.by : 8;
    if (cudaGetDevice(&b->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev) != cudaSuccess)
        return bail(CMX_ECUDA);
    int occ = batch_blocks_per_sm(nsub, b->bx, b->by);
    if (occ <= 0) return bail(CMX_EINVAL);
    if (b->cfg.blocks_per_sm > 0) occ = std::min(occ, b->cfg.blocks_per_sm);
    const int G = occ * b->nsm;

    // layouts
    b->inst.resize(n);
    long long maxc = 0;
    for (int i = 0; i < n; i++) {
        Inst &I = b->inst[i];
        const cmx_instance &d = in[i];
        I.grid = d.grid;
        I.mat = d.mat;
        I.N = d.modes.n_modes;
        I.T = d.T;
        for (int k = 0; k < I.N; k++) {
            I.omega[k] = d.modes.omega[k];
            I.kappa[k] = d.modes.kappa[k];
            I.gre[k] = d.modes.g_re[k];
            I.gim[k] = d.modes.g_im[k];
        }
        build_layout(I.lay, d.grid.nx, d.grid.ny, d.grid.nz, d.mask);
        if (I.lay.ncell_mag == 0) return bail(CMX_EINVAL);
        b->cells += I.lay.ncell_mag;
        maxc = std::max<long long>(maxc, I.lay.ncell_mag);
    }
    // team size: smallest power of two for which the largest instance fits the average load
    int K = b->cfg.team;
    if (K <= 0) {
        K = 1;
        while (K < 64 && K * 2 <= G && (double)maxc > (double)b->cells * K / G) K *= 2;
    }
    K = std::max(1, std::min(K, G));
    b->team = K;
    b->teams = G / K;
    b->blocks = b->teams * K;
    // partitions and queues (longest first onto the least loaded team)
    for (Inst &I : b->inst)
        if (!build_segments(build_columns(I.lay, b->bx, b->by), K, I.segs, I.begin))
            return bail(CMX_EINVAL);   // too many tile columns for a team of K blocks
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return b->inst[a].lay.ncell_mag > b->inst[c].lay.ncell_mag;
    });
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int t = 0; t < b->teams; t++) heap.push({0, t});
    std::vector<std::vector<int>> q(b->teams);
    for (int i : order) {
        Load l = heap.top();
        heap.pop();
        q[l.second].push_back(i);
        l.first += b->inst[i].lay.ncell_mag;
        heap.push(l);
    }
    std::vector<int> queue, qbegin{0};
    for (auto &v : q) {
        queue.insert(queue.end(), v.begin(), v.end());
        qbegin.push_back((int)queue.size());
    }

    // pool sizes
    const int nq = 3 * nsub;
    const int lc = std::max(1, solver->log_cap), tc = std::max(1, solver->trace_cap);
    size_t nf = 0, nrows = 0, nint = 0, nact = 0, nseg = 0, nlog = 0, nlogd = 0,
           ntrd = 0, maxbox = 0;
    for (Inst &I : b->inst) {
        const size_t nc = up64((size_t)I.lay.ncell);
        for (int s = 0; s < 2; s++) I.o_m[s] = nf, nf += nq * nc;
        for (int j = 0; j < 7; j++) I.o_k[j] = nf, nf += nq * nc;
        for (int j = 0; j < 2; j++) I.o_msv[j] = nf, nf += nq * nc;
        I.o_es = nf, nf += nq * nc;
        I.o_rows = nrows, nrows += I.lay.rows.size();
        I.o_box = nint, nint += I.lay.ncell;
        I.o_begin = nint, nint += I.begin.size();
        I.has_act = I.lay.padded;
        if (I.has_act) I.o_act = nact, nact += ((size_t)I.lay.ncell + 31) / 32;
        I.o_seg = nseg, nseg += I.segs.size();
        const int Q = 2 * std::max(1, I.N);
        I.o_log = nlog, nlog += lc;
        I.o_loga = nlogd, nlogd += 2 * (size_t)lc * Q;
        I.o_tr = ntrd, ntrd += tc + 2 * (size_t)tc * Q;
        maxbox = std::max(maxbox, (size_t)I.grid.nx * I.grid.ny * I.grid.nz);
    }
    if (balloc(&b->fpool, nf) || balloc(&b->rows, nrows) || balloc(&b->ipool, nint) ||
        balloc(&b->act, nact) || balloc(&b->segs, nseg) || balloc(&b->ctls, (size_t)n) ||
        balloc(&b->ctlp, (size_t)n) ||
        balloc(&b->log, nlog) || balloc(&b->logd, nlogd) || balloc(&b->trd, ntrd) ||
        balloc(&b->ctx, (size_t)n) || balloc(&b->queue, queue.size()) ||
        balloc(&b->qbegin, qbegin.size()) || balloc(&b->pending, 1) ||
        balloc(&b->dense, (size_t)nq * maxbox) ||
        cudaMallocHost((void **)&b->pending_h, sizeof(int)) != cudaSuccess)
        return bail(CMX_ENOMEM);
    b->dense_cap = (size_t)nq * maxbox;
    cudaMemset(b->fpool, 0, nf * sizeof(float));

    // uploads, contexts and initial states
    std::vector<Ctx> hctx(n);
    std::vector<Ctl *> hctlp(n);
    const double mu0 = 4.0e-7 * M_PI;
    for (int i = 0; i < n; i++) {
        Inst &I = b->inst[i];
        const size_t nc = (size_t)I.lay.ncell, nbox = (size_t)I.grid.nx * I.grid.ny * I.grid.nz;
        cudaMemcpy(b->rows + I.o_rows, I.lay.rows.data(), I.lay.rows.size() * sizeof(int2),
                   cudaMemcpyHostToDevice);
        cudaMemcpy(b->ipool + I.o_box, I.lay.box_of_cell.data(), nc * sizeof(int),
                   cudaMemcpyHostToDevice);
        cudaMemcpy(b->ipool + I.o_begin, I.begin.data(), I.begin.size() * sizeof(int),
                   cudaMemcpyHostToDevice);
        cudaMemcpy(b->segs + I.o_seg, I.segs.data(), I.segs.size() * sizeof(int4),
                   cudaMemcpyHostToDevice);
        if (I.has_act) {
            const std::vector<uint32_t> bits = active_bits(I.lay);
            cudaMemcpy(b->act + I.o_act, bits.data(), bits.size() * sizeof(uint32_t),
                       cudaMemcpyHostToDevice);
        }
        // initial magnetisation, compacted and normalised on the host; component q of a
        // compact array starts at q * stride (stride = the padded cell count)
        const size_t stride = up64(nc);
        std::vector<float> m0((size_t)nq * stride, 0.f);
        for (size_t c = 0; c < nc; c++) {
            if (!I.lay.active[c]) continue;
            for (int s = 0; s < nsub; s++) {
                float v[3] = {0.f, 0.f, s == 0 ? 1.f : -1.f};
                if (in[i].m0)
                    for (int k = 0; k < 3; k++)
                        v[k] = in[i].m0[(size_t)(3 * s + k) * nbox + I.lay.box_of_cell[c]];
                const float r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                const float r = r2 > 0.f ? 1.f / std::sqrt(r2) : 0.f;
                for (int k = 0; k < 3; k++) m0[(size_t)(3 * s + k) * stride + c] = v[k] * r;
            }
        }
        cudaMemcpy(b->fpool + I.o_m[0], m0.data(), m0.size() * sizeof(float),
                   cudaMemcpyHostToDevice);
        Ctl cl;
        memset(&cl, 0, sizeof cl);
        cl.t = 0.0;
        cl.T = I.T;
        cl.dt = solver->dt0;
        for (int q2 = 0; q2 < 2 * I.N; q2++) cl.a[q2] = in[i].a0 ? in[i].a0[q2] : 0.0;
        for (int j = 0; j < 7; j++) cl.kphys[j] = j;
        cl.skip_block = -1;
        cl.max_launch_attempts = 1;
        cudaMemcpy(b->ctls + i, &cl, sizeof cl, cudaMemcpyHostToDevice);
        hctlp[i] = b->ctls + i;

        Ctx &c = hctx[i];
        memset(&c, 0, sizeof c);
        c.nx = I.grid.nx;
        c.ny = I.grid.ny;
        c.nz = I.grid.nz;
        c.nsub = nsub;
        c.nmodes = I.N;
        c.ncell = I.lay.ncell;
        c.ncell_mag = I.lay.ncell_mag;
        c.rows = b->rows + I.o_rows;
        c.active = I.lay.holes ? b->act + I.o_act : nullptr;   // the row spans exclude padding
        c.tiles = b->segs + I.o_seg;
        c.seg_begin = b->ipool + I.o_begin;
        c.ntiles = (int)I.segs.size();
        c.u = nullptr;
        // the compact arrays use a padded stride; all stage code indexes with c.ncell, so give
        // every component its own padded slice by using the padded count as the stride
        c.m[0] = b->fpool + I.o_m[0];
        c.m[1] = b->fpool + I.o_m[1];
        for (int j = 0; j < 7; j++) c.k[j] = b->fpool + I.o_k[j];
        for (int j = 0; j < 2; j++) c.msv[j] = b->fpool + I.o_msv[j];
        c.es = b->fpool + I.o_es;
        const double exch = 2.0 * I.mat.Aex / I.mat.Ms;
        c.wx = (float)(exch / (I.grid.cx * I.grid.cx));
        c.wy = (float)(exch / (I.grid.cy * I.grid.cy));
        c.wz = (float)(exch / (I.grid.cz * I.grid.cz));
        c.anis = (float)(2.0 * I.mat.Ku / I.mat.Ms);
        for (int k = 0; k < 3; k++) {
            c.ku[k] = (float)I.mat.ku_axis[k];
            c.B0[k] = (float)I.mat.B0[k];
            c.dmg[k] = (float)(mu0 * I.mat.Ms * I.mat.Ndemag[k]);
        }
        c.BE = nsub == 2 ? (float)I.mat.BE : 0.f;
        c.pre = (float)(-I.mat.gamma / (1.0 + I.mat.alpha * I.mat.alpha));
        c.alpha = (float)I.mat.alpha;
        for (int k = 0; k < I.N; k++) {
            c.omega[k] = I.omega[k];
            c.kappa[k] = I.kappa[k];
            c.gre[k] = I.gre[k];
            c.gbre[k] = I.gre[k];   // reciprocal coupling
            c.gim[k] = I.gim[k];
            c.gbim[k] = I.gim[k];
        }
        c.two_over_gamma = 2.0 / I.mat.gamma;
        c.inv_nmag = 1.0 / (double)I.lay.ncell_mag;
        c.red_scale = overlap_scale((double)I.lay.ncell_mag);   // no profiles: |u| = 1
        c.umax = 1.f;
        c.rtol = solver->rtol;
        c.a_ref = solver->a_ref;
        c.dt_min = solver->dt_min;
        c.dt_max = solver->dt_max;
        c.sample_dt = solver->sample_dt;
        c.ctl = b->ctls + i;
        c.log = b->log + I.o_log;
        const int Q = 2 * std::max(1, I.N);
        c.log_a = b->logd + I.o_loga;
        c.log_mm = b->logd + I.o_loga + (size_t)lc * Q;
        c.log_cap = solver->log_cap;
        c.tr_t = b->trd + I.o_tr;
        c.tr_a = b->trd + I.o_tr + tc;
        c.tr_mm = b->trd + I.o_tr + tc + (size_t)tc * Q;
        c.tr_cap = solver->trace_cap;
        c.timeout_ns = 2000000000LL;
        c.stage_only = 0;
    }
    // the stage code indexes component q of a compact array at q * ncell: with the padded
    // allocation above each component slice starts at a multiple of the padded count, so the
    // stride passed to the kernels must be the padded count
    for (int i = 0; i < n; i++) hctx[i].ncell = (int)up64((size_t)b->inst[i].lay.ncell);
    cudaMemcpy(b->ctx, hctx.data(), n * sizeof(Ctx), cudaMemcpyHostToDevice);
    cudaMemcpy(b->ctlp, hctlp.data(), n * sizeof(Ctl *), cudaMemcpyHostToDevice);
    cudaMemcpy(b->queue, queue.data(), queue.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(b->qbegin, qbegin.data(), qbegin.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(CMX_ECUDA);
    *out = b;
    return CMX_OK;
}

int cmx_batch_destroy(cmx_batch *b)
{
    if (!b) return CMX_EINVAL;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return CMX_OK;
}

int cmx_batch_launch(cmx_batch *b, int n_attempts)
{
    if (!b || n_attempts <= 0) return bfail(b, CMX_EINVAL, "bad argument");
    return run_once(b, n_attempts);
}

int cmx_batch_stats(cmx_batch *b, int i, cmx_stats *st)
{
    if (!b || i < 0 || i >= b->n || !st) return bfail(b, CMX_EINVAL, "bad argument");
    Ctl c;
    int rc = read_ctl(b, i, &c);
    if (rc) return rc;
    st->t = c.t;
    st->dt = c.dt;
    st->attempts = c.attempts;
    st->accepted = c.accepted;
    st->cell_stage_updates = c.rhs_evals * (long long)b->inst[i].lay.ncell_mag;
    st->status = c.status;
    st->launches = (int)b->launches;
    return CMX_OK;
}

int cmx_batch_run(cmx_batch *b, long long max_attempts, cmx_stats *total)
{
    if (!b) return CMX_EINVAL;
    const int per_launch = 512;
    long long done_attempts = 0;
    for (;;) {
        int a = per_launch;
        if (max_attempts > 0) {
            if (done_attempts >= max_attempts) break;
            a = (int)std::min<long long>(a, max_attempts - done_attempts);
        }
        int rc = run_once(b, a);
        if (rc) return rc;
        BCU(cudaStreamSynchronize(b->stream));
        done_attempts += a;
        if (*b->pending_h == 0) break;
    }
    std::vector<Ctl> c(b->n);
    BCU(cudaMemcpy(c.data(), b->ctls, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost));
    int first_err = CMX_OK;
    if (total) {
        memset(total, 0, sizeof *total);
        total->t = INFINITY;
    }
    for (int i = 0; i < b->n; i++) {
        if (c[i].status && !first_err) {
            first_err = c[i].status;
            bfail(b, c[i].status, "instance %d: device status %d (%s)", i, c[i].status,
                  cmx_status_string(c[i].status));
        }
        if (total) {
            total->t = std::min(total->t, c[i].t);
            total->attempts += c[i].attempts;
            total->accepted += c[i].accepted;
            total->cell_stage_updates += c[i].rhs_evals * (long long)b->inst[i].lay.ncell_mag;
            if (!total->status) total->status = c[i].status;
        }
    }
    if (total) total->launches = (int)b->launches;
    return first_err;
}

int cmx_batch_spectrum(cmx_batch *b, int mode, double f0, double df, int nf, double t_start,
                       double *out)
{
    if (!b || !out || mode < 0 || mode >= MAXN || nf <= 0 || !(df > 0))
        return bfail(b, CMX_EINVAL, "bad argument");
    if (b->sv.trace_cap <= 0 || !(b->sv.sample_dt > 0))
        return bfail(b, CMX_EINVAL, "the spectral map needs traces (trace_cap, sample_dt)");
    const int tc = std::max(1, b->sv.trace_cap);
    std::vector<SpecInst> hs(b->n);
    for (int i = 0; i < b->n; i++) {
        const Inst &I = b->inst[i];
        const int Q = 2 * std::max(1, I.N);
        hs[i].t = b->trd + I.o_tr;
        hs[i].a = b->trd + I.o_tr + tc;
        hs[i].ctl = b->ctls + i;
        hs[i].q = Q;
        hs[i].cap = tc;
        hs[i].re = mode < I.N ? 2 * mode : -1;
    }
    SpecInst *ds = nullptr;
    double *dout = nullptr;
    BCU(balloc(&ds, (size_t)b->n));
    if (balloc(&dout, (size_t)b->n * nf) != cudaSuccess) {
        cudaFree(ds);
        return bfail(b, CMX_ENOMEM, "spectrum buffer");
    }
    cudaError_t e = cudaMemcpyAsync(ds, hs.data(), b->n * sizeof(SpecInst),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = launch_batch_spectrum(ds, b->n, f0, df, nf, t_start, dout, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, dout, (size_t)b->n * nf * sizeof(double), cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(ds);
    cudaFree(dout);
    if (e != cudaSuccess) return bfail(b, CMX_ECUDA, "spectrum: %s", cudaGetErrorString(e));
    return CMX_OK;
}

int cmx_batch_set_drive(cmx_batch *b, const double *eta_re, const double *eta_im, int n_eta,
                        double t0, double sigma)
{
    if (!b) return CMX_EINVAL;
    if (eta_re && (!eta_im || n_eta < 0 || n_eta > MAXN || !(sigma > 0) || !std::isfinite(t0)))
        return bfail(b, CMX_EINVAL,
                      "drive: eta_im, 0 <= n_eta <= %d, sigma > 0 and a finite t0 are needed", MAXN);
    DriveArgs d{};
    d.on = eta_re ? 1 : 0;
    for (int q = 0; q < n_eta && eta_re; q++) {
        d.re[q] = eta_re[q];
        d.im[q] = eta_im[q];
    }
    d.t0 = t0;
    d.inv_sigma = eta_re ? 1.0 / sigma : 0.0;
    BCU(launch_batch_drive(b->ctx, b->n, d, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    return CMX_OK;
}

int cmx_batch_autotune(const cmx_instance *inst, int n, const cmx_solver *solver, int sample,
                       int attempts, void *stream, cmx_batch_config *cfg, double *us,
                       int *ncand)
{
    if (!inst || n <= 0 || !solver || !cfg || attempts <= 0) return CMX_EINVAL;
    if (sample <= 0) sample = n;
    const int k = (n + sample - 1) / sample;
    std::vector<cmx_instance> sub;
    for (int i = 0; i < n; i += k) sub.push_back(inst[i]);
    const int nsub = inst[0].grid.nsub;
    const int win[2][2] = {{32, 8}, {32, 4}};
    const int teams[6] = {0, 1, 2, 4, 8, 16};
    cmx_solver sv = *solver;
    sv.log_cap = 0;
    sv.trace_cap = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CMX_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CMX_ECUDA;
    }
    double best = 1e300;
    cmx_batch_config bestc = *cfg;
    int c = 0;
    for (int w = 0; w < 2; w++)
        for (int t = 0; t < 6; t++, c++) {
            double v = NAN;
            cmx_batch_config tc = *cfg;
            tc.bx = win[w][0];
            tc.by = win[w][1];
            tc.team = teams[t];
            cmx_batch *b = nullptr;
            if (cmx_batch_create(sub.data(), (int)sub.size(), &sv, &tc, stream, &b) == CMX_OK) {
                if (run_once(b, 1) == CMX_OK && cudaEventRecord(e0, st) == cudaSuccess &&
                    run_once(b, attempts) == CMX_OK && cudaEventRecord(e1, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    std::vector<Ctl> cl(b->n);
                    bool ok = cudaMemcpy(cl.data(), b->ctls, b->n * sizeof(Ctl),
                                         cudaMemcpyDeviceToHost) == cudaSuccess;
                    for (const Ctl &x : cl) ok = ok && x.status == 0;
                    if (ok) v = 1e3 * ms;
                    if (ok && v < best && tc.team == 0) tc.team = b->team;
                    if (ok && v < best) {
                        best = v;
                        bestc = tc;
                    }
                }
                cmx_batch_destroy(b);
            }
            if (us) us[c] = v;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ncand) *ncand = c;
    if (!(best < 1e300)) return CMX_ECUDA;
    *cfg = bestc;
    return CMX_OK;
}

int cmx_batch_get_a(cmx_batch *b, int i, double *a)
{
    if (!b || i < 0 || i >= b->n || !a) return bfail(b, CMX_EINVAL, "bad argument");
    Ctl c;
    int rc = read_ctl(b, i, &c);
    if (rc) return rc;
    for (int q = 0; q < 2 * b->inst[i].N; q++) a[q] = c.a[q];
    return CMX_OK;
}

int cmx_batch_get_m(cmx_batch *b, int i, float *m)
{
    if (!b || i < 0 || i >= b->n || !m) return bfail(b, CMX_EINVAL, "bad argument");
    Ctl c;
    int rc = read_ctl(b, i, &c);
    if (rc) return rc;
    const Inst &I = b->inst[i];
    const int nq = 3 * b->nsub;
    const long long nbox = (long long)I.grid.nx * I.grid.ny * I.grid.nz;
    const int stride = (int)up64((size_t)I.lay.ncell);
    BCU(cudaMemsetAsync(b->dense, 0, (size_t)nq * nbox * sizeof(float), b->stream));
    // one component at a time (the compact slices are padded)
    for (int q = 0; q < nq; q++)
        bscatter_kernel<<<std::min<long long>(4096, (I.lay.ncell + 255) / 256), 256, 0,
                          b->stream>>>(b->fpool + I.o_m[c.mcur] + (size_t)q * stride,
                                       b->dense + (size_t)q * nbox, b->ipool + I.o_box,
                                       I.has_act ? b->act + I.o_act : nullptr, I.lay.ncell, nbox,
                                       1);
    BCU(cudaGetLastError());
    BCU(cudaMemcpyAsync(m, b->dense, (size_t)nq * nbox * sizeof(float), cudaMemcpyDeviceToHost,
                        b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    return CMX_OK;
}

int cmx_batch_get_log(cmx_batch *b, int i, cmx_step *dst, double *a, double *mm, int cap,
                      long long *n)
{
    if (!b || i < 0 || i >= b->n || cap < 0) return bfail(b, CMX_EINVAL, "bad argument");
    Ctl c;
    int rc = read_ctl(b, i, &c);
    if (rc) return rc;
    if (n) *n = c.log_n;
    const Inst &I = b->inst[i];
    const int Q = 2 * std::max(1, I.N), lc = std::max(1, b->sv.log_cap);
    const long long k = std::min<long long>({(long long)cap, c.log_n, (long long)b->sv.log_cap});
    if (k > 0) {
        if (dst) BCU(cudaMemcpy(dst, b->log + I.o_log, k * sizeof(cmx_step), cudaMemcpyDeviceToHost));
        if (a && I.N)
            BCU(cudaMemcpy(a, b->logd + I.o_loga, k * Q * sizeof(double), cudaMemcpyDeviceToHost));
        if (mm && I.N)
            BCU(cudaMemcpy(mm, b->logd + I.o_loga + (size_t)lc * Q, k * Q * sizeof(double),
                           cudaMemcpyDeviceToHost));
    }
    return CMX_OK;
}

int cmx_batch_get_trace(cmx_batch *b, int i, double *t, double *a, double *mm, int cap,
                        long long *n)
{
    if (!b || i < 0 || i >= b->n || cap < 0) return bfail(b, CMX_EINVAL, "bad argument");
    Ctl c;
    int rc = read_ctl(b, i, &c);
    if (rc) return rc;
    if (n) *n = c.trace_n;
    const Inst &I = b->inst[i];
    const int Q = 2 * std::max(1, I.N), tc = std::max(1, b->sv.trace_cap);
    const long long k = std::min<long long>({(long long)cap, c.trace_n, (long long)b->sv.trace_cap});
    if (k > 0) {
        if (t) BCU(cudaMemcpy(t, b->trd + I.o_tr, k * sizeof(double), cudaMemcpyDeviceToHost));
        if (a && I.N)
            BCU(cudaMemcpy(a, b->trd + I.o_tr + tc, k * Q * sizeof(double),
                           cudaMemcpyDeviceToHost));
        if (mm && I.N)
            BCU(cudaMemcpy(mm, b->trd + I.o_tr + tc + (size_t)tc * Q, k * Q * sizeof(double),
                           cudaMemcpyDeviceToHost));
    }
    return CMX_OK;
}

int cmx_batch_info(const cmx_batch *b, int *teams, int *team_size, int *blocks,
                   long long *cells, int *graph)
{
    if (!b) return CMX_EINVAL;
    if (teams) *teams = b->teams;
    if (team_size) *team_size = b->team;
    if (blocks) *blocks = b->blocks;
    if (cells) *cells = b->cells;
    if (graph) *graph = b->graph_ok;
    return CMX_OK;
}

}  // extern "C"
