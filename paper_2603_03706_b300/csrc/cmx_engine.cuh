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

// Per-component cavity constants: LC doubles per real component (see component_constants).
constexpr int LC = 10;

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
    double mc[MC * MAXN];                // mode constants (see MC)
    double lc[LC][2 * MAXN];             // per-component cavity constants (component_constants)
    double hw[7][6];                     // h a_Sj of the current attempt (rows S-1 = 2..6)
    double rs;                           // fixed-point overlap sum -> <m^->: 1 / (scale N_c)
    float rtolf, inv_rtolf, areff;       // error-norm constants in FP32
    float tscale;                        // per-thread fixed-point scale of the overlap partials
    int tshift;                          // block sum (units 2^-20 / tscale) -> units 1 / red_scale
    int has_kerr, has_split;
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

// Drive share eta exp(-(t - t0)^2 / (2 sigma^2)) of a component's cavity slope (out of line like
// the pump term, which keeps the FP64 exponential out of the controller's inlined code).
static __device__ __noinline__ double drive_term(double eta, double t, double t0, double inv_sigma)
{
    const double xe = (t - t0) * inv_sigma;
    return eta * exp(-0.5 * xe * xe);
}

// Parametric pump coefficient Q = P e^{-i wp t} = (qr, qi) at time t.
__device__ __forceinline__ void pump_coefficient(double pr, double pi, double pw, double t,
                                                 double &qr, double &qi)
{
    double sn, cs;
    sincos(pw * t, &sn, &cs);
    qr = pr * cs + pi * sn;
    qi = pi * cs - pr * sn;
}

// The pump's share s qi x - qr x' of component q's cavity slope (s = +1 for the real part, -1 for
// the imaginary part; x, x' the component's and its partner's cavity values).  Out of line: with
// the FP64 sine and cosine inlined into the controller, every stage kernel ran about twice as slow
// on the multimode sphere even with no pump set (measured on B300).
static __device__ __noinline__ double pump_term(double pr, double pi, double pw, double t, int q,
                                                double x, double xo)
{
    double qr, qi;
    pump_coefficient(pr, pi, pw, t, qr, qi);
    return fma((q & 1) ? -qi : qi, x, -qr * xo);
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
            if (c.has_pump) {   // -i Q conj(a) = (qi ar - qr ai, -(qr ar + qi ai))
                double qr, qi;
                pump_coefficient(L.lc[7][2 * n], L.lc[8][2 * n], L.lc[9][2 * n], ts, qr, qi);
                const double yr = y[2 * n], yi = y[2 * n + 1];
                dr += qi * yr - qr * yi;
                di -= qr * yr + qi * yi;
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

// Cavity constants of real component q = 2n + c of mode n (c = 0: real part, 1: imaginary
// part), with the sign s = +1 / -1 of the component folded in.  Lane q then forms its component
// of the slope of Eq. (12), (19) with the self-Kerr term from its own and its partner's values,
//     d_q = -kappa x + s (w + K |a|^2) x' - s g_r y' - g_i y,
// x, x' the cavity values and y, y' the overlaps of lane q and of its partner q ^ 1.  lc[5] is
// the lane's share of the feedback coefficient (2/gamma) Re[gb~ a] (pair sum of lc[5] x) and
// lc[6] the drive amplitude of the component; lc[7..9] the mode's pump Re P, Im P and frequency.
__device__ __forceinline__ void component_constants(const Ctx &c, int q, Local &L)
{
    double v[MC];
    mode_constants(c, q >> 1, v);
    const int n = q >> 1;
    double dre = c.drive_re[0], dim = c.drive_im[0];
    double pr = c.pump_re[0], pi = c.pump_im[0], pw = c.pump_w[0];
#pragma unroll
    for (int u = 1; u < MAXN; u++)
        if (n == u) {
            dre = c.drive_re[u];
            dim = c.drive_im[u];
            pr = c.pump_re[u];
            pi = c.pump_im[u];
            pw = c.pump_w[u];
        }
    L.lc[7][q] = pr;
    L.lc[8][q] = pi;
    L.lc[9][q] = pw;
    const bool im = q & 1;
    L.lc[0][q] = -v[1];
    L.lc[1][q] = im ? -v[0] : v[0];
    L.lc[2][q] = im ? v[2] : -v[2];
    L.lc[3][q] = -v[3];
    L.lc[4][q] = im ? -v[6] : v[6];
    L.lc[5][q] = c.two_over_gamma * (im ? -v[5] : v[4]);
    L.lc[6][q] = im ? dim : dre;
}

// Cavity value a_S of stage S of the current attempt, one real component per lane of warp 0
// (lane q < 2N when `own`), and the feedback coefficient of each mode, hrf_n = (2/gamma)
// Re[gb~_n a_{n,S}] (Eq. (5), (13)), as the sum over the mode's two lanes.  Called by all lanes
// of warp 0.  One FP64 instruction per slope: the weights h a_Sj come from the attempt's table.
template <int S>
__device__ __forceinline__ void cavity_stage_value(Local &L, Coef &cf, int q, bool own)
{
    double v = 0.0;
    if (own) {
        v = L.a[q];
#pragma unroll
        for (int j = 0; j < S - 1; j++)
            if (dp_a(S - 1, j) != 0.0)
                v += (S == 2 ? L.h * dp_a(1, 0) : L.hw[S - 1][j]) * L.ka[j][q];
        L.as[q] = v;
    }
    double p = own ? L.lc[5][q] * v : 0.0;
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    if (own && !(q & 1)) cf.hrf[q >> 1] = (float)p;
}

// The weights h a_Sj of the whole attempt, entry q of rows S = 2..7, in FP64 for the cavity and
// FP32 for the magnet's stage combination; run by 36 threads once the attempt's size is known
// (the coefficient is selected, then multiplied once).
__device__ __forceinline__ void attempt_coefficients(Coef &cf, Local &L, double h, int q)
{
    double a = 0.0;
#pragma unroll
    for (int s = 1; s < 7; s++)
#pragma unroll
        for (int j = 0; j < 6; j++)
            if (q == (s - 1) * 6 + j) a = dp_a(s, j);
    const double w = h * a;
    L.hw[1 + q / 6][q % 6] = w;
    cf.cf[1 + q / 6][q % 6] = (float)w;
}

// Work after the barrier of stage S, on warp 0 (the caller's block barrier follows).  Lane
// q < 2N owns real component q = 2n + c of mode n: from its grid sum (fixed point, `sq`) it
// forms its component of the overlap <m^->_n (Eq. (18)) and of the cavity slope (Eq. (12),
// (19), with the drive and the Kerr term), its adjoint stores and, before stage 7, its component
// of the next stage's cavity value.  After stage 7 the lanes take the scaled error norm (FP32,
// warp maximum) and the accept decision, each lane the same, and update their own components of
// the state; lane 0 keeps the scalar part (time, counters, step size, log).  Only the team's
// rank 0 writes log, trace and adjoint stores.  An FP64 warp instruction occupies the FP64 pipe
// for tens of cycles on this GPU whatever the number of active lanes, so the part is written
// for few FP64 instructions (one component per lane, per-lane constants, no block barrier).
//
// The controller in two parts: controller_cavity<S> is the cavity work of stage S (everything of
// stages 1..6; at stage 7 the cavity slope k_7 and the scaled cavity error norm, which need no
// magnet data), controller_decide the accept decision of stage 7, which needs the magnet's error
// maximum.  Both run on all lanes of warp 0; controller<S> runs them back to back, the
// single-block integrator overlaps the first with the magnet's last pass.
struct Cav7 {
    double y, d;   // the lane's overlap component and cavity slope of stage 7
    float e2;      // scaled cavity error norm (every lane)
};

template <int S>
__device__ __forceinline__ Cav7 controller_cavity(const Ctx &c, const Team &tm, Local &L,
                                                  Coef &cf, long long sq)
{
    const int N = c.nmodes;
    const int q = threadIdx.x;
    __syncwarp();   // the lanes' shuffles below need the whole warp at the same point
    const bool own = q < 2 * N;
    const bool rec = tm.rank == 0;
    const double y = own ? (double)sq * L.rs : 0.0;
    const double yo = __shfl_xor_sync(0xffffffffu, y, 1);
    double d = 0.0;
    if (own) {
        const double x = L.as[q], xo = L.as[q ^ 1];
        double t = L.lc[1][q];
        if (L.has_kerr) t = fma(L.lc[4][q], fma(x, x, xo * xo), t);
        d = L.lc[0][q] * x;
        d = fma(t, xo, d);
        d = fma(L.lc[2][q], yo, d);
        d = fma(L.lc[3][q], y, d);
        if (L.has_split && !L.replay) {   // operator split: cavity held during magnet steps
            d = 0.0;
        } else {
            // drive and parametric pump at this stage's time t + c_S h
            const double ts = S == 1 ? L.t : L.t + dp_c(S - 1) * L.h;
            if (c.has_drive) d += drive_term(L.lc[6][q], ts, c.drive_t0, c.drive_inv_sigma);
            if (c.has_pump)   // -i Q conj(a): component q gets s qi x - qr x', s = +1 / -1
                d += pump_term(L.lc[7][q], L.lc[8][q], L.lc[9][q], ts, q, x, xo);
        }
        L.mm[q] = y;
        L.ka[S - 1][q] = d;
        if (rec) {
            // adjoint stores: a rejected attempt's checkpoint is overwritten by the accepted retry
            const int slot = checkpoint_slot<S>(c, L);
            if (slot >= 0 && c.traj_a) {
                double *dd = c.traj_a + (size_t)slot * traj_stride(N);
                dd[q] = S == 7 ? L.as[q] : L.a[q];
                dd[2 * N + q] = d;
                dd[4 * N + q] = y;
                if (q == 0) dd[6 * N] = S == 7 ? (L.last ? L.T : L.t + L.h) : L.t;
            }
            if (c.rec_a && L.replay && L.replay_pos < c.rec_steps) {
                double *dd = c.rec_a + ((size_t)L.replay_pos * 7 + (S - 1)) * 4 * N;
                dd[q] = L.as[q];
                dd[2 * N + q] = y;
                if (S == 2 && q == 0 && c.rec_t) c.rec_t[L.replay_pos] = L.t;
            }
        }
        if (S == 1) L.mm_n[q] = y;
    }
    if (S >= 2 && S < 7) cavity_stage_value<(S < 7 ? S + 1 : 7)>(L, cf, q, own);
    if (S != 7) {
        if (q == 0) {
            L.rhs_evals += 1;
            if (S == 1) {
                L.k1_valid = 1;
                if (c.stage_only) L.done = 1;
            }
        }
        if (S == 1 && L.has_split && L.split_pending && !c.stage_only && !L.replay) {
            // cavity step over the coming interval with the overlaps of the current m; the
            // slope just computed used the old feedback field: evaluate stage 1 again
            __syncwarp();
            if (q == 0) {
                split_cavity_step(c, L, L.mm);
                L.split_pending = 0;
                L.k1_valid = 0;
            }
        }
        return Cav7{0.0, 0.0, 0.f};
    }

    // stage 7: error estimate of the lane's component; magnitudes in FP32 (they only scale the
    // error norm), maxima over lanes 0 .. 2 MAXN - 1 (lanes >= 2N hold 0, NaN propagates)
    double e = 0.0;
    if (own) {
#pragma unroll
        for (int j = 0; j < 7; j++)
            if (dp_e(j) != 0.0) e += dp_e(j) * (j == 6 ? d : L.ka[j][q]);
    }
    const float ef = (float)e, af = own ? (float)L.a[q] : 0.f, sf = own ? (float)L.as[q] : 0.f;
    const float efo = __shfl_xor_sync(0xffffffffu, ef, 1);
    const float afo = __shfl_xor_sync(0xffffffffu, af, 1);
    const float sfo = __shfl_xor_sync(0xffffffffu, sf, 1);
    float en = own ? cf.h * hypotf(ef, efo) : 0.f;
    float an = own ? fmaxf(hypotf(af, afo), hypotf(sf, sfo)) : 0.f;
#pragma unroll
    for (int o = MAXN; o > 0; o >>= 1) {
        en = nanmax(en, __shfl_xor_sync(0xffffffffu, en, o));
        an = fmaxf(an, __shfl_xor_sync(0xffffffffu, an, o));
    }
    // scaled error norm: magnet max-norm against rtol, cavity against rtol max(a_ref, |a|)
    return Cav7{y, d, en / (L.rtolf * fmaxf(L.areff, an))};
}

__device__ __forceinline__ void controller_decide(const Ctx &c, const Team &tm, Local &L,
                                                  const Cav7 &v, float emax)
{
    const int N = c.nmodes;
    const int q = threadIdx.x;
    const bool own = q < 2 * N;
    const bool rec = tm.rank == 0;
    const long long li = L.log_n;
    const double y = v.y, d = v.d;
    const float e1 = emax * L.inv_rtolf;
    const float e2 = v.e2;
    const float err = (e1 > e2 || e1 != e1) ? e1 : e2;
    const bool finite = isfinite(err);
    const int accepted = finite && L.status == 0 && (L.replay || err <= 1.f);
    const double h = L.h, t0 = L.t;
    __syncwarp();
    if (q == 0) {
        L.attempts += 1;
        L.launch_attempts += 1;
        if (!finite) {
            L.status = CMX_ENAN;
            L.done = 1;
        }
        const double t1 = L.last ? L.T : (L.at_split ? L.split_next : t0 + h);
        // uniform trace: cubic Hermite for a_n (end slopes k1, k7), linear for <m^->_n; it
        // reads the state at t0, which the lanes replace only after this block
        if (accepted && c.tr_cap > 0 && c.sample_dt > 0.0) {
            long long tn = L.trace_n;
            double ts = L.trace_next;
            while (tn < c.tr_cap && ts <= t1) {
                const double th = (ts - t0) / h;
                const double h00 = (2 * th - 3) * th * th + 1, h10 = ((th - 2) * th + 1) * th;
                const double h01 = (3 - 2 * th) * th * th, h11 = (th - 1) * th * th;
                if (rec) {
                    c.tr_t[tn] = ts;
                    for (int k = 0; k < 2 * N; k++) {
                        c.tr_a[tn * 2 * N + k] = h00 * L.a[k] + h10 * h * L.ka[0][k] +
                                                 h01 * L.as[k] + h11 * h * L.ka[6][k];
                        c.tr_mm[tn * 2 * N + k] = (1 - th) * L.mm_n[k] + th * L.mm[k];
                    }
                }
                tn++;
                ts += c.sample_dt;
            }
            L.trace_n = tn;
            L.trace_next = ts;
        }
        if (rec && li < c.log_cap) {
            cmx_step st;
            st.t = accepted ? t1 : t0;
            st.dt = h;
            st.err = (double)err;
            st.accepted = accepted;
            st.pad = 0;
            c.log[li] = st;
        }
        L.log_n = li + 1;
        L.rhs_evals += 1;
        if (accepted) {
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
        if (L.replay) {
            L.replay_pos += 1;
            if (L.replay_pos >= L.replay_n || L.t >= L.T) L.done = 1;
        } else if (L.status == 0) {
            // step factor 0.9 err^(-1/5) clamped to [0.2, 5], in FP32 (FP64 pow has a very long
            // latency here); the clamp bounds themselves are exact in FP64
            const float ff = err > 0.f ? 0.9f * powf(err, -0.2f) : 5.f;
            double fac = ff >= 5.f ? 5.0 : (ff < 0.2f ? 0.2 : (double)ff);
            if (accepted) {
                if (L.last_rejected && ff > 1.f) fac = 1.0;
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
        // t reaches T only through an accepted last step (attempt_size lands it on T)
        if ((accepted && L.last) || L.launch_attempts >= L.max_launch_attempts) L.done = 1;
    }
    __syncwarp();
    if (own && accepted) {   // the accepted step's state, FSAL slope and log entry of component q
        if (rec && li < c.log_cap) {
            c.log_a[li * 2 * N + q] = L.as[q];
            c.log_mm[li * 2 * N + q] = y;
        }
        L.a[q] = L.as[q];
        L.ka[0][q] = d;
        L.mm_n[q] = y;
    }
}

template <int S>
__device__ __forceinline__ void controller(const Ctx &c, const Team &tm, Local &L, Coef &cf,
                                           long long sq, float emax)
{
    if (threadIdx.x >= 32) return;
    const Cav7 v = controller_cavity<S>(c, tm, L, cf, sq);
    if (S == 7) controller_decide(c, tm, L, v, emax);
}

// Block sum of the per-thread overlap accumulators and block max of |e_m|, added into
// accumulator set `set` of the control block.  Each thread scales its FP32 partials by L.tscale
// (a power of two that keeps a partial below 2^24 in magnitude) and splits each into two int32
// digits, the integer part and the remainder in units of 2^-20; a warp sums each digit exactly in
// one redux instruction, the block in int64, and the total is added into the grid's fixed-point
// sum (scale red_scale), so it does not depend on the order of the blocks.  A partial outside
// the range (an unstable or non-finite state) sets range_error, which the controller turns into
// CMX_ENAN.  The maximum goes through an integer max on the bit pattern of the non-negative
// float (NaN is largest).
template <class SM>
__device__ void block_reduce(const Ctx &c, const Team &tm, SM &sm, const Acc &acc, int set,
                             const Local &L)
{
    const int NT = blockDim.x, NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float ts = L.tscale;
    bool bad = false;
#pragma unroll
    for (int n = 0; n < MAXN; n++) {
        if (n >= c.nmodes) break;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float v = (k ? acc.im[n] : acc.re[n]) * ts;
            bad |= !(fabsf(v) <= 16777216.f);
            const float vh = rintf(v);   // exact below 2^24; v - vh is exact as well
            const int dh = __reduce_add_sync(0xffffffffu, __float2int_rn(vh));
            const int dl = __reduce_add_sync(0xffffffffu, __float2int_rn((v - vh) * 1048576.f));
            if (lane == 0) {
                sm.red[warp][2 * n + k].hi = __int_as_float(dh);
                sm.red[warp][2 * n + k].lo = __int_as_float(dl);
            }
        }
    }
    const unsigned e = __reduce_max_sync(0xffffffffu, __float_as_uint(acc.emax));
    if (lane == 0) sm.redmax[warp] = __uint_as_float(e);
    if (bad) atomicExch(&c.ctl->range_error, 1);
    __syncthreads();
    const int Q = 2 * c.nmodes;
    if (threadIdx.x < Q) {
        long long sh = 0, sl = 0;
        for (int w = 0; w < NW; w++) {
            sh += __float_as_int(sm.red[w][threadIdx.x].hi);
            sl += __float_as_int(sm.red[w][threadIdx.x].lo);
        }
        long long v = sh * (1ll << 20) + sl;   // units of 2^-20 / tscale
        const int d = L.tshift;                  // to units of 1 / red_scale
        v = d >= 0 ? v * (1ll << d) : (v + (1ll << (-d - 1))) >> (-d);
        atomicAdd(reinterpret_cast<unsigned long long *>(&c.ctl->racc[set][threadIdx.x]),
                  (unsigned long long)v);
    }
    if (threadIdx.x == NT - 1) {
        unsigned m = 0u;
        for (int w = 0; w < NW; w++) m = max(m, __float_as_uint(sm.redmax[w]));
        atomicMax(&c.ctl->remax[set], m);
    }
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

}  // namespace cmx

#include "cmx_demag.cuh"

namespace cmx {

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
// (right after its barrier), which also formed this stage's cavity value; the first two stages
// of an attempt form it here (and at stage 2 the weights h a_Sj of the whole attempt).
// After the barrier the component lanes read the grid sums of set `set` (identical for every
// block), this stage starts the next one's copies (S < 7), so that the read latency and the
// controller overlap the first copies, and warp 0 runs the controller.  The team's rank 0
// clears the set that stage count + 2 will use: every block read it before arriving at this
// barrier.
template <int S, bool FD, class SM>
__device__ bool run_stage(const Ctx &c, const Team &tm, SM &sm, Local &L, Coef &cf, Pipe &pp,
                          bool begun)
{
    const int tid = threadIdx.x, N = c.nmodes;
    const float *mn = L.mcur ? c.m[1] : c.m[0];
    float *mnew = L.mcur ? c.m[0] : c.m[1];
    // with full demag (kernels compiled with FD) the stage's copies start after its demag passes
    // (they use the pool)
    const bool fd = FD && c.fd;
    begun = begun && !fd;
    if (!begun) {
        if (tid < 7) sm.kp[tid] = slope_buffer(c, L.kphys[tid]);
        __syncthreads();
        if (!fd) stage_begin<S>(c, sm, mn, pp);
    }
    if (S <= 2) {
        if (tid < 32) cavity_stage_value<S>(L, cf, tid, tid < 2 * N);
        if (S == 2 && tid >= 32 && tid < 32 + 36) attempt_coefficients(cf, L, L.h, tid - 32);
        if (S == 2 && tid == 96) cf.h = (float)L.h;
        __syncthreads();
    }
    if constexpr (FD) {
        if (fd) {
            if (!demag_field<S>(c, tm, sm, L, cf, mn)) return false;
            stage_begin<S>(c, sm, mn, pp);
        }
    }
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
    block_reduce(c, tm, sm, acc, set, L);
    if (!grid_barrier<SM>(c, tm, L, S)) return false;
    long long sq = 0;
    float emax = 0.f;
    {
        const volatile Ctl *g = c.ctl;
        if (tid < 2 * N) sq = g->racc[set][tid];
        if (S == 7 && tid < 32) {
            const unsigned bits = g->remax[set];
            emax = g->range_error ? __int_as_float(0x7fffffff) : __uint_as_float(bits);
        }
        if (tm.rank == 0 && tid >= 32 && tid <= 32 + 2 * N) {
            volatile Ctl *w = c.ctl;
            const int clr = (set + 2) % 3, q = tid - 32;
            if (q < 2 * N) w->racc[clr][q] = 0;
            else w->remax[clr] = 0u;
        }
    }
    if (S >= 2 && S < 7 && !c.stage_only && !fd) stage_begin<(S < 7 ? S + 1 : 7)>(c, sm, mn, pp);
    controller<S>(c, tm, L, cf, sq, emax);
    __syncthreads();
    return true;
}

// Integrate one problem with a team of blocks: load the problem's state into the block's copy,
// this block's segments and the mode constants, then run Dormand-Prince attempts until the
// problem is done (t >= T, replay end, attempt budget of the launch, or an error).  The team's
// rank-0 block writes the state back.  Returns false if the run stopped on a device error.
template <bool FD = false, class SM>
__device__ bool integrate(const Ctx &c, const Team &tm, SM &sm, Local &L, Coef &cf, int &s_stop)
{
    if (threadIdx.x == 0) {
        load_local(c, L);
        L.rs = c.inv_nmag / c.red_scale;   // exact: the scale is a power of two
        L.rtolf = (float)c.rtol;
        L.inv_rtolf = (float)(1.0 / c.rtol);
        L.areff = (float)c.a_ref;
        int hk = 0;
#pragma unroll
        for (int u = 0; u < MAXN; u++)
            if (u < c.nmodes && c.kerr[u] != 0.0) hk = 1;
        L.has_kerr = hk;
        L.has_split = c.split_dt > 0.0;
    }
    if (threadIdx.x < 2 * c.nmodes) component_constants(c, threadIdx.x, L);
    if (threadIdx.x >= 32 && threadIdx.x < 39) cf.e[threadIdx.x - 32] = (float)dp_e(threadIdx.x - 32);
    if (threadIdx.x < c.nmodes) mode_constants(c, threadIdx.x, L.mc + MC * threadIdx.x);
    {
        const int sb = __ldg(&c.seg_begin[tm.rank]), se = __ldg(&c.seg_begin[tm.rank + 1]);
        const bool ok = idx_ok(c, se - sb, MAX_BLOCK_SEGMENTS + 1, 11) &&
                        idx_ok(c, sb, (long long)c.ntiles + 1, 12) &&
                        idx_ok(c, se, (long long)c.ntiles + 1, 13);
        const int n = ok ? se - sb : 0;
        if (threadIdx.x == 0) sm.nseg = n;
        for (int t = threadIdx.x; t < n; t += blockDim.x) sm.seg[t] = __ldg(&c.tiles[sb + t]);
    }
    __syncthreads();
    stage_cache_rows(c, sm);
    if (threadIdx.x == 0) {
        // fixed-point scale of this block's overlap partials: a thread computes at most P cells
        // per stage (interior planes of the block's segments), each contributing at most
        // |u| |m| <= 2 umax
        int P = 0;
        for (int t = 0; t < sm.nseg; t++) P += sm.seg[t].w - sm.seg[t].z;
        P *= cells_per_thread(&sm);
        const float bound = 2.f * (float)(P > 1 ? P : 1) * fmaxf(c.umax, 1.f);
        const int k = 24 - (int)ceilf(log2f(bound));
        L.tscale = ldexpf(1.f, k);
        L.tshift = ilogb(c.red_scale) - k - 20;
    }
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
            if (!(ok = run_stage<1, FD>(c, tm, sm, L, cf, pp, false)))
                break;
            if (c.stage_only) break;
        }
        if (!ok || c.stage_only) break;
        if (!(ok = run_stage<2, FD>(c, tm, sm, L, cf, pp, false))) break;
        if (!(ok = run_stage<3, FD>(c, tm, sm, L, cf, pp, true))) break;
        if (!(ok = run_stage<4, FD>(c, tm, sm, L, cf, pp, true))) break;
        if (!(ok = run_stage<5, FD>(c, tm, sm, L, cf, pp, true))) break;
        if (!(ok = run_stage<6, FD>(c, tm, sm, L, cf, pp, true))) break;
        if (!(ok = run_stage<7, FD>(c, tm, sm, L, cf, pp, true))) break;
    }
    if (ok && tm.rank == 0 && threadIdx.x == 0) store_local(c, L);
    __syncthreads();
    return ok;
}

}  // namespace cmx
