// Device engine of the integrator (sm_103a): per-block integrator state, cavity update and
// step-size controller, team barrier and reductions, one Dormand-Prince stage, and the attempt
// loop over a problem.  Used by the single-problem kernel and by the batched kernel.
//
// Every Dormand-Prince attempt runs inside one persistent launch with a barrier after each stage:
// the cavity slope of a stage needs the overlap reduction over all cells (Eq. (18)).  The
// barrier is a monotonic arrival counter of the team (one release-atomic per block, acquire
// polling).  Before arriving, every block adds its overlap sums into the team's accumulators as
// fixed-point integers (exact, so the totals do not depend on the order of arrival); after it
// every block reads the same totals and runs the same FP64 cavity update and step-size
// controller on its own shared-memory copy of the integrator state: identical inputs and
// identical code give every block the same decision, deterministic from run to run.  The team's block 0 records the step
// log and the trace and writes the state back.  No step returns to the host (Sec. III A).
#pragma once

#include "cmx_stage.cuh"

namespace cmx {

// The blocks that integrate one problem together: this block's rank among them, their count and
// their arrival counter.  A single-problem launch is one team of all blocks.
struct Team {
    int rank, nblk;
    unsigned *bar;
};

// Block-local copy of the integrator state.
struct Local {
    double t, dt, T, h;
    double a[2 * MAXN];
    double ka[7][2 * MAXN];
    double mm_n[2 * MAXN];
    double trace_next;
    double split_next, split_t0;
    long long split_k;
    int split_pending, at_split;
    long long attempts, accepted, launch_attempts, max_launch_attempts, rhs_evals;
    long long replay_pos, replay_n, log_n, trace_n;
    const double *replay_dts;
    double mm[2 * MAXN], as[2 * MAXN];   // overlaps and cavity stage value of this stage
    double err_n[MAXN], amax_n[MAXN];    // per-mode error and amplitude (stage 7)
    double mc[MC * MAXN];                // mode constants (see MC)
    unsigned bar_target;                 // arrival count that completes the next barrier
    int skip_block;
    int kphys[7];
    int mcur, k1_valid, last_rejected, last, replay, done, status;
};

__device__ __forceinline__ void load_local(const Ctx &c, Local &L)
{
    const volatile Ctl *g = c.ctl;
    L.t = g->t;
    L.dt = g->dt;
    L.T = g->T;
    for (int q = 0; q < 2 * c.nmodes; q++) {
        L.a[q] = g->a[q];
        L.mm_n[q] = g->mm_n[q];
        for (int j = 0; j < 7; j++) L.ka[j][q] = g->ka[j][q];
    }
    L.trace_next = g->trace_next;
    L.split_next = g->split_next;
    L.split_t0 = g->split_t0;
    L.split_k = g->split_k;
    L.split_pending = g->split_pending;
    L.at_split = 0;
    L.attempts = g->attempts;
    L.accepted = g->accepted;
    L.launch_attempts = g->launch_attempts;
    L.max_launch_attempts = g->max_launch_attempts;
    L.rhs_evals = g->rhs_evals;
    L.replay_pos = g->replay_pos;
    L.replay_n = g->replay_n;
    L.log_n = g->log_n;
    L.trace_n = g->trace_n;
    L.replay_dts = g->replay_dts;
    for (int j = 0; j < 7; j++) L.kphys[j] = g->kphys[j];
    L.mcur = g->mcur;
    L.k1_valid = g->k1_valid;
    L.last_rejected = g->last_rejected;
    L.replay = g->replay;
    L.done = g->done;
    L.status = g->status;
    L.last = 0;
    L.h = 0.0;
    L.bar_target = 0;
    L.skip_block = g->skip_block;
}

__device__ __forceinline__ void store_local(const Ctx &c, const Local &L)
{
    volatile Ctl *g = c.ctl;
    g->t = L.t;
    g->dt = L.dt;
    for (int q = 0; q < 2 * c.nmodes; q++) {
        g->a[q] = L.a[q];
        g->mm_n[q] = L.mm_n[q];
        for (int j = 0; j < 7; j++) g->ka[j][q] = L.ka[j][q];
    }
    g->trace_next = L.trace_next;
    g->split_next = L.split_next;
    g->split_k = L.split_k;
    g->split_pending = L.split_pending;
    g->attempts = L.attempts;
    g->accepted = L.accepted;
    g->launch_attempts = L.launch_attempts;
    g->rhs_evals = L.rhs_evals;
    g->replay_pos = L.replay_pos;
    g->log_n = L.log_n;
    g->trace_n = L.trace_n;
    for (int j = 0; j < 7; j++) g->kphys[j] = L.kphys[j];
    g->mcur = L.mcur;
    g->k1_valid = L.k1_valid;
    g->last_rejected = L.last_rejected;
    g->done = L.done;
    if (L.status) atomicCAS(&c.ctl->status, 0, L.status);
    __threadfence();
}

// Size of the next attempt: the replay list, or min(dt, dt_max) shortened to land on T (and,
// in the operator-split scheme, on the next interval boundary).
__device__ __forceinline__ void attempt_size(const Ctx &c, Local &L)
{
    L.last = 0;
    L.at_split = 0;
    if (L.replay) {
        L.h = L.replay_dts[L.replay_pos];
        return;
    }
    L.h = L.dt < c.dt_max ? L.dt : c.dt_max;
    if (L.t + L.h >= L.T) {
        L.h = L.T - L.t;
        L.last = 1;
    }
    if (c.split_dt > 0.0 && L.t + L.h >= L.split_next) {
        L.h = L.split_next - L.t;
        L.at_split = 1;
        L.last = L.split_next >= L.T;
    }
}

// Checkpoint slot that stage S of the current attempt writes, or -1: stage 1 of the first
// attempt writes slot 0 (the initial state and its slope), stage 7 writes slot k when the
// attempt would complete k * traj_every accepted steps.
template <int S>
__device__ __forceinline__ int checkpoint_slot(const Ctx &c, const Local &L)
{
    if (!c.traj_m || (S != 1 && S != 7)) return -1;
    const long long k = L.accepted - c.traj_base;
    long long slot = -1;
    if (S == 1 && k == 0) slot = 0;
    if (S == 7 && (k + 1) % c.traj_every == 0) slot = (k + 1) / c.traj_every;
    return slot < c.traj_slots ? (int)slot : -1;
}

// Cavity right-hand side (-i w - kappa) a + i g~ mm - i K |a|^2 a for one mode (Eq. (12), (19),
// with the optional self-Kerr term); the mode constants come from the block's shared copy.
__device__ __forceinline__ void cavity_rhs(const double *mc, int n, double ar, double ai,
                                           double mr, double mi, double &dr, double &di)
{
    const double *q = mc + MC * n;
    const double w = q[0], k = q[1], gr = q[2], gi = q[3], K = q[6];
    const double pr = gr * mr - gi * mi, pi = gr * mi + gi * mr;   // g~ <m^->
    const double k2 = K * (ar * ar + ai * ai);
    dr = -k * ar + w * ai - pi + k2 * ai;
    di = -k * ai - w * ar + pr - k2 * ar;
}

// Operator-split scheme: one classical RK4 step of the cavity from L.t to the next boundary
// with the overlaps held at mm (those of the current magnetisation), on 2N real components,
// run by one thread.  Same slope as cavity_rhs plus the drive.
static __device__ __noinline__ void split_cavity_step(const Ctx &c, Local &L, const double *mm)
{
    const int N = c.nmodes;
    const double h = L.split_next - L.t;
    double a0[2 * MAXN], y[2 * MAXN], acc[2 * MAXN], k[2 * MAXN];
    for (int q = 0; q < 2 * N; q++) a0[q] = y[q] = L.a[q];
    for (int st = 0; st < 4; st++) {
        const double ts = L.t + (st == 0 ? 0.0 : (st == 3 ? h : 0.5 * h));
        double env = 0.0;
        if (c.has_drive) {
            const double x = (ts - c.drive_t0) * c.drive_inv_sigma;
            env = exp(-0.5 * x * x);
        }
        for (int n = 0; n < N; n++) {
            double dr, di;
            cavity_rhs(L.mc, n, y[2 * n], y[2 * n + 1], mm[2 * n], mm[2 * n + 1], dr, di);
            if (c.has_drive) {
                double er = c.drive_re[0], ei = c.drive_im[0];
                for (int u = 1; u < MAXN; u++)
                    if (n == u) {
                        er = c.drive_re[u];
                        ei = c.drive_im[u];
                    }
                dr += er * env;
                di += ei * env;
            }
            k[2 * n] = dr;
            k[2 * n + 1] = di;
        }
        const double wgt = (st == 0 || st == 3) ? 1.0 : 2.0;
        for (int q = 0; q < 2 * N; q++) {
            acc[q] = (st == 0 ? 0.0 : acc[q]) + wgt * k[q];
            if (st < 3) y[q] = a0[q] + (st == 2 ? h : 0.5 * h) * k[q];
        }
    }
    for (int q = 0; q < 2 * N; q++) L.a[q] = a0[q] + h / 6.0 * acc[q];
}

// Stage-S cavity update and, after stage 7, error norm, accept/reject and step-size control,
// on the block's copy L.  L.as holds the cavity stage value a_S (set before the stage), `sum`
// the grid sums of the overlaps and `emax` the grid maximum of |e_m|.  The per-mode FP64 work
// runs on 2N threads; the decision itself on thread 0.  Only block 0 writes log and trace.
template <int S>
__device__ void controller(const Ctx &c, const Team &tm, Local &L, const double *sum, float emax)
{
    const int N = c.nmodes;
    const int tid = threadIdx.x;
    if (tid < 2 * N) L.mm[tid] = sum[tid] * c.inv_nmag;
    __syncthreads();
    if (tid < N) {
        double dr, di;
        cavity_rhs(L.mc, tid, L.as[2 * tid], L.as[2 * tid + 1], L.mm[2 * tid],
                   L.mm[2 * tid + 1], dr, di);
        if (c.split_dt > 0.0 && !L.replay) {   // operator split: cavity held during magnet steps
            dr = 0.0;
            di = 0.0;
        } else if (c.has_drive) {   // the drive at this stage's time t + c_S h
            const double ts = S == 1 ? L.t : L.t + dp_c(S - 1) * L.h;
            const double x = (ts - c.drive_t0) * c.drive_inv_sigma;
            const double env = exp(-0.5 * x * x);
            double er = c.drive_re[0], ei = c.drive_im[0];
#pragma unroll
            for (int u = 1; u < MAXN; u++)
                if (tid == u) {
                    er = c.drive_re[u];
                    ei = c.drive_im[u];
                }
            dr += er * env;
            di += ei * env;
        }
        L.ka[S - 1][2 * tid] = dr;
        L.ka[S - 1][2 * tid + 1] = di;
        if (S == 7) {
            double er = 0.0, ei = 0.0;
#pragma unroll
            for (int j = 0; j < 7; j++) {
                const double kr = j == 6 ? dr : L.ka[j][2 * tid];
                const double ki = j == 6 ? di : L.ka[j][2 * tid + 1];
                er += dp_e(j) * kr;
                ei += dp_e(j) * ki;
            }
            // magnitudes in FP32: they only scale the error norm
            L.err_n[tid] = (double)(fabsf((float)L.h) * hypotf((float)er, (float)ei));
            L.amax_n[tid] = (double)fmaxf(hypotf((float)L.a[2 * tid], (float)L.a[2 * tid + 1]),
                                          hypotf((float)L.as[2 * tid], (float)L.as[2 * tid + 1]));
        }
    }
    __syncthreads();
    if (tid != 0) return;
    L.rhs_evals += 1;
    if (tm.rank == 0) {
        // adjoint stores: a rejected attempt's checkpoint is overwritten by the accepted retry
        const int slot = checkpoint_slot<S>(c, L);
        if (slot >= 0 && c.traj_a) {
            double *d = c.traj_a + (size_t)slot * traj_stride(N);
            for (int q = 0; q < 2 * N; q++) {
                d[q] = S == 7 ? L.as[q] : L.a[q];
                d[2 * N + q] = L.ka[S - 1][q];
                d[4 * N + q] = L.mm[q];
            }
            d[6 * N] = S == 7 ? (L.last ? L.T : L.t + L.h) : L.t;
        }
        if (c.rec_a && L.replay && L.replay_pos < c.rec_steps) {
            double *d = c.rec_a + ((size_t)L.replay_pos * 7 + (S - 1)) * 4 * N;
            for (int q = 0; q < 2 * N; q++) {
                d[q] = L.as[q];
                d[2 * N + q] = L.mm[q];
            }
        }
    }
    if (S == 1) {
        L.k1_valid = 1;
        for (int q = 0; q < 2 * N; q++) L.mm_n[q] = L.mm[q];
        if (c.stage_only) L.done = 1;
        if (c.split_dt > 0.0 && L.split_pending && !c.stage_only && !L.replay) {
            // cavity step over the coming interval with the overlaps of the current m; the
            // slope just computed used the old feedback field: evaluate stage 1 again
            split_cavity_step(c, L, L.mm);
            L.split_pending = 0;
            L.k1_valid = 0;
        }
        return;
    }
    if (S != 7) return;

    // scaled error norm
    const double h = L.h;
    double ea = 0.0, amax = 0.0;
    for (int n = 0; n < N; n++) {
        if (L.err_n[n] > ea || L.err_n[n] != L.err_n[n]) ea = L.err_n[n];
        amax = fmax(amax, L.amax_n[n]);
    }
    const double e1 = (double)emax / c.rtol;
    const double e2 = ea / (c.rtol * fmax(c.a_ref, amax));
    const double err = (e1 > e2 || e1 != e1) ? e1 : e2;
    if (!isfinite(err)) {
        L.status = CMX_ENAN;
        L.done = 1;
    }
    const int accepted = L.status == 0 && (L.replay || err <= 1.0);
    const bool rec = tm.rank == 0;
    const long long li = L.log_n;
    L.attempts += 1;
    L.launch_attempts += 1;
    const double t0 = L.t;
    double t1 = t0;
    const double *as = L.as, *mm = L.mm;
    if (accepted) {
        t1 = L.last ? L.T : (L.at_split ? L.split_next : t0 + h);
        // uniform trace: cubic Hermite for a_n (end slopes k1, k7), linear for <m^->_n
        if (c.tr_cap > 0 && c.sample_dt > 0.0) {
            long long tn = L.trace_n;
            double ts = L.trace_next;
            while (tn < c.tr_cap && ts <= t1) {
                const double th = (ts - t0) / h;
                const double h00 = (2 * th - 3) * th * th + 1, h10 = ((th - 2) * th + 1) * th;
                const double h01 = (3 - 2 * th) * th * th, h11 = (th - 1) * th * th;
                if (rec) {
                    c.tr_t[tn] = ts;
                    for (int q = 0; q < 2 * N; q++) {
                        c.tr_a[tn * 2 * N + q] = h00 * L.a[q] + h10 * h * L.ka[0][q] +
                                                 h01 * as[q] + h11 * h * L.ka[6][q];
                        c.tr_mm[tn * 2 * N + q] = (1 - th) * L.mm_n[q] + th * mm[q];
                    }
                }
                tn++;
                ts += c.sample_dt;
            }
            L.trace_n = tn;
            L.trace_next = ts;
        }
        for (int q = 0; q < 2 * N; q++) {
            L.a[q] = as[q];
            L.ka[0][q] = L.ka[6][q];
            L.mm_n[q] = mm[q];
        }
        const int k0 = L.kphys[0];
        L.kphys[0] = L.kphys[6];
        L.kphys[6] = k0;
        L.mcur ^= 1;
        L.t = t1;
        L.accepted += 1;
        if (L.at_split && t1 < L.T) {   // boundary reached: cavity step before the next interval
            L.split_k += 1;
            L.split_next = fmin(L.split_t0 + (double)(L.split_k + 1) * c.split_dt, L.T);
            L.split_pending = 1;
            L.k1_valid = 0;
        }
    }
    if (rec && li < c.log_cap) {
        cmx_step st;
        st.t = accepted ? t1 : t0;
        st.dt = h;
        st.err = err;
        st.accepted = accepted;
        st.pad = 0;
        c.log[li] = st;
        if (accepted)
            for (int q = 0; q < 2 * N; q++) {
                c.log_a[li * 2 * N + q] = as[q];
                c.log_mm[li * 2 * N + q] = mm[q];
            }
    }
    L.log_n = li + 1;

    if (L.replay) {
        L.replay_pos += 1;
        if (L.replay_pos >= L.replay_n) L.done = 1;
    } else if (L.status == 0) {
        // step factor in FP32 (FP64 pow has a very long latency here)
        const float ef = (float)err;
        double fac = ef > 0.f ? (double)(0.9f * powf(ef, -0.2f)) : 5.0;
        fac = fmin(5.0, fmax(0.2, fac));
        if (accepted) {
            if (L.last_rejected && fac > 1.0) fac = 1.0;
            L.last_rejected = 0;
            L.dt = fmin(h * fac, c.dt_max);
        } else {
            L.last_rejected = 1;
            L.dt = h * fac;
            if (L.dt < c.dt_min) {
                L.status = CMX_ESTEPFAIL;
                L.done = 1;
            }
        }
    }
    if (L.t >= L.T || L.launch_attempts >= L.max_launch_attempts) L.done = 1;
}

// Block sum of the per-thread overlap accumulators (compensated pairs, fixed shuffle order)
// and block max of |e_m|, added into accumulator set `set` of the control block: the sums as
// fixed-point integers (exact, so their total does not depend on the order of the blocks), the
// maximum through an integer max on the bit pattern of the non-negative float.
template <class SM>
__device__ void block_reduce(const Ctx &c, const Team &tm, SM &sm, const Acc &acc, int set)
{
    const int NT = blockDim.x, NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int n = 0; n < MAXN; n++) {
        if (n >= c.nmodes) break;
        F2 r = {acc.re[n], 0.f}, i = {acc.im[n], 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r = f2_add(r, f2_shfl_xor(r, o));
            i = f2_add(i, f2_shfl_xor(i, o));
        }
        if (lane == 0) {
            sm.red[warp][2 * n] = r;
            sm.red[warp][2 * n + 1] = i;
        }
    }
    float e = acc.emax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = nanmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) sm.redmax[warp] = e;
    __syncthreads();
    const int Q = 2 * c.nmodes;
    if (threadIdx.x < Q) {
        F2 s = {0.f, 0.f};
        for (int w = 0; w < NW; w++) s = f2_add(s, sm.red[w][threadIdx.x]);
        const double v = ((double)s.hi + (double)s.lo) * c.red_scale;
        if (fabs(v) < 4.0e18) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&c.ctl->racc[set][threadIdx.x]),
                      (unsigned long long)__double2ll_rn(v));
        } else {
            atomicExch(&c.ctl->range_error, 1);
        }
    }
    if (threadIdx.x == NT - 1) {
        float m = 0.f;
        for (int w = 0; w < NW; w++) m = nanmax(m, sm.redmax[w]);
        atomicMax(&c.ctl->remax[set], __float_as_uint(m));
    }
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// After the barrier: the grid sums of set `set`, identical for every block.  The team's rank 0
// then clears the set that stage count + 2 will use (every block has finished reading it: it
// was read before the arrival at this barrier).
template <class SM>
__device__ void grid_reduce(const Ctx &c, const Team &tm, SM &sm, double *out, float *emax, int set)
{
    const int Q = 2 * c.nmodes;
    volatile Ctl *g = c.ctl;
    if ((int)threadIdx.x < Q) out[threadIdx.x] = (double)g->racc[set][threadIdx.x] / c.red_scale;
    if ((int)threadIdx.x == Q) {
        const unsigned bits = g->remax[set];
        *emax = g->range_error ? __int_as_float(0x7fffffff) : __uint_as_float(bits);
    }
    if (tm.rank == 0) {
        const int clr = (set + 2) % 3;
        if ((int)threadIdx.x < Q) g->racc[clr][threadIdx.x] = 0;
        if ((int)threadIdx.x == Q) g->remax[clr] = 0u;
    }
    __syncthreads();
}

// Team barrier: every block of the team adds 1 to a monotonic arrival counter with release
// semantics and polls it with acquire loads until all blocks of this barrier have arrived.
// Waits are bounded by c.timeout_ns: on time-out the block sets CMX_ETIMEOUT and the run stops.
// The block's accumulator additions were issued before the __syncthreads that precedes the
// release-add.  Returns false if the run must stop.
template <class SM>
__device__ bool grid_barrier(const Ctx &c, const Team &tm, Local &L, int where)
{
    __shared__ int s_ok;
    Ctl *ctl = c.ctl;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        if (L.skip_block == tm.rank) {
            s_ok = -1;   // test hook: leave without arriving
        } else {
            L.bar_target += tm.nblk;
            red_add_release(tm.bar, 1u);
            const unsigned long long t0 = global_timer_ns();
            unsigned spins = 0;
            while ((int)(ld_acquire(tm.bar) - L.bar_target) < 0) {
                if ((++spins & 31u) == 0) {
                    if (ld_volatile_int(&ctl->status) != 0) {
                        s_ok = 0;
                        break;
                    }
                    if (global_timer_ns() - t0 > (unsigned long long)c.timeout_ns) {
                        atomicCAS(&ctl->status, 0, (int)CMX_ETIMEOUT);
                        ctl->timeout_where = where;
                        s_ok = 0;
                        break;
                    }
                }
            }
        }
    }
    __syncthreads();
    return s_ok > 0;
}

// Physical buffer of logical slope j (select rather than index the kernel-parameter array,
// which keeps it out of local memory).
__device__ __forceinline__ const float *slope_buffer(const Ctx &c, int kj)
{
    const float *p = c.k[0];
#pragma unroll
    for (int u = 1; u < 7; u++)
        if (kj == u) p = c.k[u];
    return p;
}

// One stage.  If `begun`, the copy pipeline of this stage was started by the previous stage
// (right after its barrier).  After the barrier this stage starts the next one (S < 7) before
// it reduces the partials and updates the cavity, so those latencies overlap the first copies.
template <int S, class SM>
__device__ bool run_stage(const Ctx &c, const Team &tm, SM &sm, Local &L, Coef &cf,
                          double *s_sum, float *s_emax, Pipe &pp, bool begun)
{
    const int tid = threadIdx.x, N = c.nmodes;
    const double h = L.h;
    const float *mn = L.mcur ? c.m[1] : c.m[0];
    float *mnew = L.mcur ? c.m[0] : c.m[1];
    if (!begun) {
        if (tid < 7) sm.kp[tid] = slope_buffer(c, L.kphys[tid]);
        __syncthreads();
        stage_begin<S>(c, sm, mn, pp);
    }
    // cavity stage value a_S = a_n + h sum_j a_Sj k^a_j (FP64, one thread per real component)
    if (tid < 2 * N) {
        double v = L.a[tid];
#pragma unroll
        for (int j = 0; j < S - 1; j++)
            if (dp_a(S - 1, j) != 0.0) v += h * dp_a(S - 1, j) * L.ka[j][tid];
        L.as[tid] = v;
    }
    if (tid >= 32 && tid < 38) cf.cf[tid - 32] = (float)(h * (tid - 32 < S - 1 ? dp_a(S - 1, tid - 32) : 0.0));
    if (tid >= 64 && tid < 71) cf.e[tid - 64] = (float)dp_e(tid - 64);
    if (tid == 96) cf.h = (float)h;
    __syncthreads();
    if (tid < N)
        cf.hrf[tid] = (float)(c.two_over_gamma * (L.mc[MC * tid + 4] * L.as[2 * tid] -
                                                  L.mc[MC * tid + 5] * L.as[2 * tid + 1]));
    __syncthreads();
    Acc acc;
#pragma unroll
    for (int n = 0; n < MAXN; n++) acc.re[n] = acc.im[n] = 0.f;
    acc.emax = 0.f;
    // checkpoint slot and stage-record step written by this stage (adjoint stores only)
    const int tslot = checkpoint_slot<S>(c, L);
    const int rslot = (S >= 2 && c.rec_m && L.replay && L.replay_pos < c.rec_steps)
                          ? (int)L.replay_pos : -1;
    stage_run<S>(c, sm, (float *)sm.kp[S - 1], mn, mnew, cf, pp, tslot, rslot, acc);
    const int set = (int)(L.rhs_evals % 3);
    block_reduce(c, tm, sm, acc, set);
    if (!grid_barrier<SM>(c, tm, L, S)) return false;
    if (S >= 2 && S < 7 && !c.stage_only) stage_begin<(S < 7 ? S + 1 : 7)>(c, sm, mn, pp);
    grid_reduce(c, tm, sm, s_sum, s_emax, set);
    controller<S>(c, tm, L, s_sum, *s_emax);
    __syncthreads();
    return true;
}

// Integrate one problem with a team of blocks: load the problem's state into the block's copy,
// this block's segments and the mode constants, then run Dormand-Prince attempts until the
// problem is done (t >= T, replay end, attempt budget of the launch, or an error).  The team's
// rank-0 block writes the state back.  Returns false if the run stopped on a device error.
template <class SM>
__device__ bool integrate(const Ctx &c, const Team &tm, SM &sm, Local &L, Coef &cf,
                          double *s_sum, float &s_emax, int &s_stop)
{
    if (threadIdx.x == 0) load_local(c, L);
    if (threadIdx.x < c.nmodes) mode_constants(c, threadIdx.x, L.mc + MC * threadIdx.x);
    {
        const int sb = __ldg(&c.seg_begin[tm.rank]), se = __ldg(&c.seg_begin[tm.rank + 1]);
        if (threadIdx.x == 0) sm.nseg = se - sb;
        for (int t = threadIdx.x; t < se - sb; t += blockDim.x) sm.seg[t] = __ldg(&c.tiles[sb + t]);
    }
    __syncthreads();
    stage_cache_rows(c, sm);
    __syncthreads();
    bool ok = true;
    Pipe pp;
    for (;;) {
        if (threadIdx.x == 0) {
            s_stop = L.status != 0 || L.done || ld_volatile_int(&c.ctl->status) != 0 ||
                     (c.stage_only && L.k1_valid);
            if (!s_stop) attempt_size(c, L);
        }
        __syncthreads();
        if (s_stop) break;
        while (!L.k1_valid) {   // twice at an operator-split boundary (see controller<1>)
            if (!(ok = run_stage<1>(c, tm, sm, L, cf, s_sum, &s_emax, pp, false)))
                break;
            if (c.stage_only) break;
        }
        if (!ok || c.stage_only) break;
        if (!(ok = run_stage<2>(c, tm, sm, L, cf, s_sum, &s_emax, pp, false))) break;
        if (!(ok = run_stage<3>(c, tm, sm, L, cf, s_sum, &s_emax, pp, true))) break;
        if (!(ok = run_stage<4>(c, tm, sm, L, cf, s_sum, &s_emax, pp, true))) break;
        if (!(ok = run_stage<5>(c, tm, sm, L, cf, s_sum, &s_emax, pp, true))) break;
        if (!(ok = run_stage<6>(c, tm, sm, L, cf, s_sum, &s_emax, pp, true))) break;
        if (!(ok = run_stage<7>(c, tm, sm, L, cf, s_sum, &s_emax, pp, true))) break;
    }
    if (ok && tm.rank == 0 && threadIdx.x == 0) store_local(c, L);
    __syncthreads();
    return ok;
}

}  // namespace cmx
