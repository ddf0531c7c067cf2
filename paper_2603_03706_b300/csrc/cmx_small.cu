// Single-block integrator for small grids (sm_103a).
//
// A grid of a few hundred to about a thousand magnetic cells (the 280-cell 8^3 sphere of the
// single-mode Rabi and anticrossing runs of Sec. IV A-B) is integrated by ONE block that keeps,
// for every magnetic cell, m_n and the new state, the stage value, the seven slopes, the error
// partial, the mode profiles and a neighbour table in shared memory (up to 288 cells, each
// worker's cell in its registers instead, with only the values neighbours read in shared
// memory: CellReg).  No stage touches global memory except for the step log and the trace.
//
// The block is split by warps.  Warp 0 runs the cavity update and the step-size controller (the
// engine's own, in FP64: one cavity component per lane), warp 1 (the helper) the part of the
// cavity update of stages 2..6 that needs no overlap sums (small_prepare); warps 2.. (the
// workers) own the cells.
// A stage S of the workers is two passes over their cells:
//   A  the overlap partials of the stage values m_S (Eq. (18)), summed over the block as fixed-
//      point integers (the same digits as the multi-block reduction, shared-memory atomics, so
//      the totals do not depend on the order) -> handed to warp 0;
//   B  once warp 0 has formed the stage's cavity value a_S and its feedback coefficients: the
//      field, the slope and the cell's next stage value m_{S+1} (stage 6 also the error partial,
//      stage 7 the new state and |e_m|).
// The cavity slope of stage S needs only the overlap sums of pass A, so warp 0 runs the
// controller of stage S while the workers run pass B of stage S and pass A of stage S + 1: the
// FP64 cavity work, which holds a warp for about 64 cycles per instruction, is hidden behind the
// cell passes.  Named barriers carry the hand-offs (sums ready: workers arrive, warp 0 waits;
// feedback ready: warp 0 arrives, workers wait; and between warp 0 and the helper); the
// feedback coefficients and the sums are double-buffered by stage parity.  Only the accept decision after stage 7 (which needs
// the error maximum of pass B) is a full block barrier, once per attempt.  The per-cell
// arithmetic is the tiled kernel's (cell_slope, the same combine order), so the two integrate
// the same discrete system.
#include "cmx_engine.cuh"
#include "cmx_kernels.h"

namespace cmx {

constexpr int SMALL_NT = 352;               // warp 0, warp 1 (helper), nine worker warps
constexpr int SMALL_W0 = 64;                // first worker thread
constexpr int SMALL_WK = SMALL_NT - SMALL_W0;   // worker threads (one cell each up to 288 cells)
// named barriers: warp 0 with the workers (SMALL_WK + 32 threads) and warp 0 with the helper (64)
constexpr int BAR_SUMS = 1;                 // a stage's overlap sums complete (workers arrive)
constexpr int BAR_FEED = 2;                 // a stage's feedback coefficients set (warp 0 arrives)
constexpr int BAR_PRE = 3;                  // the helper's part of a stage's cavity update ready
constexpr int BAR_HELP = 4;                 // the previous stage's cavity update done (warp 0)
constexpr int BAR_CW = SMALL_WK + 32;

size_t small_smem_bytes(int nm, int nsub, int nmodes, bool has_u)
{
    const size_t nq = 3 * (size_t)nsub;
    return ((2 + 2 + 1 + 7) * nq + (has_u ? (size_t)nmodes : 0)) * nm * sizeof(float) +
           6 * (size_t)nm * sizeof(int);
}

__device__ __forceinline__ void bar_sync_n(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void bar_arrive_n(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Block-level scratch: the two int32 digits of the fixed-point overlap sums by stage parity
// (see small_sums), the error maximum (bit pattern of a non-negative float; NaN is largest) and
// the range flag.
struct SmallRed {
    int dig[2][2 * MAXN][2];
    unsigned emax;
    int bad;
};

// Per-thread partials are scaled to at most 2^(SMALL_TBITS-1) in magnitude (a factor 2 of room
// for stage values slightly off the unit sphere); one beyond 2^SMALL_TBITS is a range error, so
// the block's integer digits stay inside int32 (SMALL_WK * 2^22 < 2^31).
constexpr int SMALL_TBITS = 22;
static_assert((long long)SMALL_WK << SMALL_TBITS < (1ll << 31), "digit sums must fit int32");

// Workers: block sums of the per-thread overlap partials of one stage into dig[par].  Each
// partial is scaled by L.tscale and split into two int32 digits (integer part and remainder in
// units of 2^-20), summed exactly over the warp (redux); lane q adds component q's two warp
// digits into the block's (integer atomics: exact, in any order).  A partial outside the range
// (an unstable or non-finite state) sets `bad`.
__device__ __forceinline__ void small_sums(const Ctx &c, const Local &L, const Acc &acc,
                                           SmallRed &R, int par)
{
    const int lane = threadIdx.x & 31;
    const float ts = L.tscale;
    bool bad = false;
#pragma unroll
    for (int n = 0; n < MAXN; n++) {
        if (n >= c.nmodes) break;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float v = (k ? acc.im[n] : acc.re[n]) * ts;
            bad |= !(fabsf(v) <= (float)(1 << SMALL_TBITS));
            const float vh = rintf(v);
            const int dh = __reduce_add_sync(0xffffffffu, __float2int_rn(vh));
            const int dl = __reduce_add_sync(0xffffffffu, __float2int_rn((v - vh) * 1048576.f));
            if (lane == 2 * n + k) {
                atomicAdd(&R.dig[par][2 * n + k][0], dh);
                atomicAdd(&R.dig[par][2 * n + k][1], dl);
            }
        }
    }
    if (bad) atomicOr(&R.bad, 1);
}

struct SmallBuf {
    float *mb0, *mb1;      // the two state buffers (index = the control block's mcur)
    float *ms[2];          // stage values: stage S reads ms[S & 1], writes m_{S+1} to the other
    float *es, *kk;        // error partial, slopes [physical][q][cell]
    const float *uu;       // profiles [n][cell]
    const int *nb;         // neighbours [-x, +x, -y, +y, -z, +z][cell], -1 = none
};

// Workers (threads SMALL_W0..): stage S of their cells (see the file comment).  `cw` holds the
// attempt's coefficients and the feedback coefficients of stage S.  Stage 1 reads m_n, stage 2
// m_2 = m_n + h a_21 k_1 (formed by the caller's pass).  Pass A reads only the worker's own
// cells, and the feedback barrier between the passes orders every worker's stage values before
// any neighbour read of pass B.  Stage 7 adds the workers' error maximum into R.emax.
template <int NS, bool HU, int S>
__device__ void small_work(const Ctx &c, int nm, const SmallBuf &b, const Local &L,
                           const Coef &cw, SmallRed &R)
{
    constexpr int NQ = 3 * NS;
    const int wt = threadIdx.x - SMALL_W0;
    const size_t V = (size_t)NQ * nm;
    const float *mn = L.mcur ? b.mb1 : b.mb0;
    float *mnew = L.mcur ? b.mb0 : b.mb1;
    const float *src = S == 1 ? mn : b.ms[S & 1];
    {   // pass A: overlap partials of the stage values, in cell_slope's order of operations
        Acc acc;
#pragma unroll
        for (int n = 0; n < MAXN; n++) acc.re[n] = acc.im[n] = 0.f;
        for (int i = wt; i < nm; i += SMALL_WK) {
            float mt[2];
#pragma unroll
            for (int k = 0; k < 2; k++)
                mt[k] = NS == 2 ? src[k * nm + i] + src[(3 + k) * nm + i] : src[k * nm + i];
            const float hx = NS == 2 ? 0.5f * mt[0] : mt[0];
            const float hy = NS == 2 ? 0.5f * mt[1] : mt[1];
#pragma unroll
            for (int n = 0; n < MAXN; n++) {
                if (n >= c.nmodes) break;
                const float un = HU ? b.uu[n * nm + i] : 1.f;
                acc.re[n] = fmaf(un, hx, acc.re[n]);
                acc.im[n] = fmaf(-un, hy, acc.im[n]);
            }
        }
        small_sums(c, L, acc, R, S & 1);
    }
    bar_arrive_n(BAR_SUMS, BAR_CW);
    bar_sync_n(BAR_FEED, BAR_CW);
    // pass B: field, slope, next stage value
    Acc acc;   // cell_slope's overlap partials are not used here (pass A formed them)
#pragma unroll
    for (int n = 0; n < MAXN; n++) acc.re[n] = acc.im[n] = 0.f;
    acc.emax = 0.f;
    float *kout = b.kk + L.kphys[S - 1] * V;
    for (int i = wt; i < nm; i += SMALL_WK) {
        int nbr[6];
#pragma unroll
        for (int d = 0; d < 6; d++) {
            nbr[d] = b.nb[d * nm + i];
            if (nbr[d] >= 0 && !idx_ok(c, nbr[d], nm, 14)) nbr[d] = -1;
        }
        const float nx_ = (float)(nbr[0] >= 0) + (float)(nbr[1] >= 0);
        const float ny_ = (float)(nbr[2] >= 0) + (float)(nbr[3] >= 0);
        const float nz_ = (float)(nbr[4] >= 0) + (float)(nbr[5] >= 0);
        float m[NS][3], B[NS][3];
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float *v = src + (s * 3 + k) * nm;
                const float cen = v[i];
                float nv[6];
#pragma unroll
                for (int d = 0; d < 6; d++) nv[d] = nbr[d] >= 0 ? v[nbr[d]] : 0.f;
                m[s][k] = cen;
                B[s][k] = c.wx * (nv[0] + nv[1] - nx_ * cen) + c.wy * (nv[2] + nv[3] - ny_ * cen) +
                          c.wz * (nv[4] + nv[5] - nz_ * cen);
            }
        float ucell[MAXN];
#pragma unroll
        for (int n = 0; n < MAXN; n++) ucell[n] = (HU && n < c.nmodes) ? b.uu[n * nm + i] : 1.f;
        const float bdem[3] = {0.f, 0.f, 0.f};   // full demag runs on the tiled kernel
        float kv[NS][3];
        cell_slope<NS, HU>(c, cw, m, B, ucell, bdem, acc, kv);
#pragma unroll
        for (int s = 0; s < NS; s++) {
#pragma unroll
            for (int k = 0; k < 3; k++) kout[(s * 3 + k) * nm + i] = kv[s][k];
            if (S >= 2 && S <= 6) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const int q = s * 3 + k;
                    float a = mn[q * nm + i], e = 0.f;
#pragma unroll
                    for (int j = 0; j < S - 1; j++) {
                        if (dp_a(S, j) == 0.0 && !(S == 6 && dp_e(j) != 0.0)) continue;
                        const float kj = b.kk[L.kphys[j] * V + q * nm + i];
                        if (dp_a(S, j) != 0.0) a = fmaf(cw.cf[S][j], kj, a);
                        if (S == 6 && dp_e(j) != 0.0) e = fmaf(cw.e[j], kj, e);
                    }
                    b.ms[(S + 1) & 1][q * nm + i] = fmaf(cw.cf[S][S - 1], kv[s][k], a);
                    if (S == 6) b.es[q * nm + i] = fmaf(cw.e[5], kv[s][k], e);
                }
            }
            if (S == 7) {
                const float *mm = m[s];
                const float r = rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const int q = s * 3 + k;
                    mnew[q * nm + i] = mm[k] * r;
                    const float e7 = cw.h * fmaf(cw.e[6], kv[s][k], b.es[q * nm + i]);
                    acc.emax = nanmax(acc.emax, fabsf(e7));
                }
            }
        }
    }
    if (S == 7) {
        const unsigned e = __reduce_max_sync(0xffffffffu, __float_as_uint(acc.emax));
        if ((threadIdx.x & 31) == 0) atomicMax(&R.emax, e);
    }
}

// Register state of a worker's cell when every worker owns at most one cell (nm <= SMALL_WK):
// the cell's m_n, current stage value, the seven slopes of the attempt by stage (k[j] = k_{j+1};
// the FSAL swap is a copy), the error partial, the normalised stage-7 value (the new state if
// the attempt is accepted), its profile values and neighbour table.  Only the stage values that
// neighbours read (and the state, for stage 1 and the write-back) go through shared memory.
template <int NS>
struct CellReg {
    float mn[3 * NS], ms[3 * NS], k[7][3 * NS], es[3 * NS], m7[3 * NS];
    float u[MAXN];
    int nbr[6];
    int mcur;
};

// small_work for one cell per worker with the cell's state in registers (see CellReg); the same
// operations in the same order as small_work.
template <int NS, bool HU, int S>
__device__ __forceinline__ void small_work_reg(const Ctx &c, int nm, const SmallBuf &b,
                                               const Local &L, const Coef &cw, SmallRed &R,
                                               CellReg<NS> &r)
{
    const int i = threadIdx.x - SMALL_W0;
    const bool own = i < nm;
    const float *mn = L.mcur ? b.mb1 : b.mb0;
    float *mnew = L.mcur ? b.mb0 : b.mb1;
    const float *src = S == 1 ? mn : b.ms[S & 1];
    const float(&mc)[3 * NS] = S == 1 ? r.mn : r.ms;   // the cell's own stage value
    {   // pass A
        Acc acc;
#pragma unroll
        for (int n = 0; n < MAXN; n++) acc.re[n] = acc.im[n] = 0.f;
        if (own) {
            float mt[2];
#pragma unroll
            for (int k = 0; k < 2; k++) mt[k] = NS == 2 ? mc[k] + mc[3 + k] : mc[k];
            const float hx = NS == 2 ? 0.5f * mt[0] : mt[0];
            const float hy = NS == 2 ? 0.5f * mt[1] : mt[1];
#pragma unroll
            for (int n = 0; n < MAXN; n++) {
                if (n >= c.nmodes) break;
                const float un = HU ? r.u[n] : 1.f;
                acc.re[n] = fmaf(un, hx, acc.re[n]);
                acc.im[n] = fmaf(-un, hy, acc.im[n]);
            }
        }
        small_sums(c, L, acc, R, S & 1);
    }
    bar_arrive_n(BAR_SUMS, BAR_CW);
    bar_sync_n(BAR_FEED, BAR_CW);
    Acc acc;
#pragma unroll
    for (int n = 0; n < MAXN; n++) acc.re[n] = acc.im[n] = 0.f;
    acc.emax = 0.f;
    if (own) {
        const float nx_ = (float)(r.nbr[0] >= 0) + (float)(r.nbr[1] >= 0);
        const float ny_ = (float)(r.nbr[2] >= 0) + (float)(r.nbr[3] >= 0);
        const float nz_ = (float)(r.nbr[4] >= 0) + (float)(r.nbr[5] >= 0);
        float m[NS][3], B[NS][3];
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float *v = src + (s * 3 + k) * nm;
                const float cen = mc[s * 3 + k];
                float nv[6];
#pragma unroll
                for (int d = 0; d < 6; d++) nv[d] = r.nbr[d] >= 0 ? v[r.nbr[d]] : 0.f;
                m[s][k] = cen;
                B[s][k] = c.wx * (nv[0] + nv[1] - nx_ * cen) + c.wy * (nv[2] + nv[3] - ny_ * cen) +
                          c.wz * (nv[4] + nv[5] - nz_ * cen);
            }
        float ucell[MAXN];
#pragma unroll
        for (int n = 0; n < MAXN; n++) ucell[n] = (HU && n < c.nmodes) ? r.u[n] : 1.f;
        const float bdem[3] = {0.f, 0.f, 0.f};
        float kv[NS][3];
        cell_slope<NS, HU>(c, cw, m, B, ucell, bdem, acc, kv);
#pragma unroll
        for (int s = 0; s < NS; s++) {
#pragma unroll
            for (int k = 0; k < 3; k++) r.k[S - 1][s * 3 + k] = kv[s][k];
            if (S >= 2 && S <= 6) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const int q = s * 3 + k;
                    float a = r.mn[q], e = 0.f;
#pragma unroll
                    for (int j = 0; j < S - 1; j++) {
                        if (dp_a(S, j) == 0.0 && !(S == 6 && dp_e(j) != 0.0)) continue;
                        const float kj = r.k[j][q];
                        if (dp_a(S, j) != 0.0) a = fmaf(cw.cf[S][j], kj, a);
                        if (S == 6 && dp_e(j) != 0.0) e = fmaf(cw.e[j], kj, e);
                    }
                    const float nxt = fmaf(cw.cf[S][S - 1], kv[s][k], a);
                    r.ms[q] = nxt;
                    b.ms[(S + 1) & 1][q * nm + i] = nxt;
                    if (S == 6) r.es[q] = fmaf(cw.e[5], kv[s][k], e);
                }
            }
            if (S == 7) {
                const float *mm = m[s];
                const float rn = rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const int q = s * 3 + k;
                    r.m7[q] = mm[k] * rn;
                    mnew[q * nm + i] = r.m7[q];
                    const float e7 = cw.h * fmaf(cw.e[6], kv[s][k], r.es[q]);
                    acc.emax = nanmax(acc.emax, fabsf(e7));
                }
            }
        }
    }
    if (S == 7) {
        const unsigned e = __reduce_max_sync(0xffffffffu, __float_as_uint(acc.emax));
        if ((threadIdx.x & 31) == 0) atomicMax(&R.emax, e);
    }
}

// Warp 0, stage S: wait for the workers' overlap sums, take component q's digits (lane q < 2N),
// clear them for stage S + 2, convert the total to the grid units 1 / red_scale and release the
// workers' pass B (the stage's feedback coefficients were set before).
template <int S>
__device__ __forceinline__ long long small_take_sums(const Ctx &c, const Local &L, SmallRed &R)
{
    const int q = threadIdx.x;
    bar_sync_n(BAR_SUMS, BAR_CW);
    long long sq = 0;
    if (q < 2 * c.nmodes) {
        const long long v = (long long)R.dig[S & 1][q][0] * (1ll << 20) + R.dig[S & 1][q][1];
        R.dig[S & 1][q][0] = 0;
        R.dig[S & 1][q][1] = 0;
        const int d = L.tshift;
        sq = d >= 0 ? v * (1ll << d) : (v + (1ll << (-d - 1))) >> (-d);
    }
    __syncwarp();
    bar_arrive_n(BAR_FEED, BAR_CW);
    return sq;
}

// Warp 0, stage S: the sums (small_take_sums), then the controller of stages 1..6, which forms
// the next stage's cavity value and feedback coefficients into cfw[(S+1)&1].  Returns the lane's
// fixed-point sum (the caller runs stage 7's controller).
template <int S>
__device__ long long small_control(const Ctx &c, Local &L, Coef *cfw, SmallRed &R)
{
    const long long sq = small_take_sums<S>(c, L, R);
    if (S < 7) {
        const Team tm{0, 1, nullptr};
        controller<S>(c, tm, L, cfw[(S + 1) & 1], sq, 0.f);
        __syncwarp();
    }
    return sq;
}

// The helper warp's part of the cavity update of stage S (2..6), the terms that do not need the
// stage's overlap sums (lane q < 2N, component q): d0 = fma(t, x', -kappa-term x) of the cavity
// slope with the Kerr-shifted frequency t, and P = a_n + sum_{j < S-1} (h a_{S+1,j}) k^a_j of
// the next stage's cavity value, in the order of operations of controller_cavity<S> and
// cavity_stage_value<S+1>, so that warp 0 finishes both with the same roundings.  An FP64 warp
// instruction occupies a warp for about 64 cycles, while four warps of an SM can run them at
// once: moving these 2 + S - 1 instructions to a second warp shortens warp 0's stage.
struct SmallPre {
    double d0[2 * MAXN], P[2 * MAXN];
};

template <int S>
__device__ void small_prepare(const Ctx &c, const Local &L, SmallPre &pre)
{
    const int q = threadIdx.x - 32;
    if (q < 2 * c.nmodes) {
        const double x = L.as[q], xo = L.as[q ^ 1];
        double t = L.lc[1][q];
        if (L.has_kerr) t = fma(L.lc[4][q], fma(x, x, xo * xo), t);
        double d = L.lc[0][q] * x;
        d = fma(t, xo, d);
        pre.d0[q] = d;
        double v = L.a[q];
#pragma unroll
        for (int j = 0; j < S - 1; j++)
            if (dp_a(S, j) != 0.0) v += L.hw[S][j] * L.ka[j][q];
        pre.P[q] = v;
    }
    __syncwarp();
    bar_arrive_n(BAR_PRE, 64);
}

// Warp 0: controller_cavity<S> for S = 2..6 of the single-block integrator (which records no
// adjoint data and has no checkpoints), finishing the helper's terms: the overlap <m^->_n of
// component q (Eq. (18)), the cavity slope (Eq. (12), (19), drive and pump), the next stage's
// cavity value and the feedback coefficients into cf.hrf.
template <int S>
__device__ void small_cavity(const Ctx &c, Local &L, Coef &cf, long long sq, const SmallPre &pre)
{
    const int N = c.nmodes;
    const int q = threadIdx.x;
    __syncwarp();
    const bool own = q < 2 * N;
    const double y = own ? (double)sq * L.rs : 0.0;
    const double yo = __shfl_xor_sync(0xffffffffu, y, 1);
    double d = 0.0;
    if (own) {
        const double x = L.as[q], xo = L.as[q ^ 1];
        d = pre.d0[q];
        d = fma(L.lc[2][q], yo, d);
        d = fma(L.lc[3][q], y, d);
        if (L.has_split && !L.replay) {
            d = 0.0;
        } else {
            const double ts = L.t + dp_c(S - 1) * L.h;
            if (c.has_drive) d += drive_term(L.lc[6][q], ts, c.drive_t0, c.drive_inv_sigma);
            if (c.has_pump) d += pump_term(L.lc[7][q], L.lc[8][q], L.lc[9][q], ts, q, x, xo);
        }
        L.mm[q] = y;
        L.ka[S - 1][q] = d;
    }
    __syncwarp();   // every lane has read the stage's cavity values before they are replaced
    double v = 0.0;
    if (own) {
        v = pre.P[q];
        v += L.hw[S][S - 1] * d;
        L.as[q] = v;
    }
    double p = own ? L.lc[5][q] * v : 0.0;
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    if (own && !(q & 1)) cf.hrf[q >> 1] = (float)p;
    if (q == 0) L.rhs_evals += 1;
}

// Warp 0, stage S = 2..6 with the helper: as small_control, with the cavity update finished from
// the helper's terms; afterwards the helper may prepare stage S + 1.
template <int S>
__device__ void small_control_pre(const Ctx &c, Local &L, Coef *cfw, SmallRed &R,
                                  const SmallPre &pre)
{
    const long long sq = small_take_sums<S>(c, L, R);
    bar_sync_n(BAR_PRE, 64);
    small_cavity<S>(c, L, cfw[(S + 1) & 1], sq, pre);
    __syncwarp();
    if (S < 6) bar_arrive_n(BAR_HELP, 64);
}

// Warp 0, before stage 2 of an attempt (its size known, k_1 valid): the cavity value a_2 and
// the feedback coefficients of stage 2 (into cfw[0]), the weights h a_Sj of the attempt and h,
// copied into both coefficient sets.
__device__ void small_attempt_setup(Local &L, Coef *cfw, int nmodes)
{
    const int q = threadIdx.x;
    cavity_stage_value<2>(L, cfw[0], q, q < 2 * nmodes);
    attempt_coefficients(cfw[0], L, L.h, q);
    if (q < 4) attempt_coefficients(cfw[0], L, L.h, q + 32);
    if (q == 0) cfw[0].h = (float)L.h;
    __syncwarp();
    float *d = &cfw[1].cf[0][0];
    const float *s = &cfw[0].cf[0][0];
    for (int k = q; k < 7 * 6; k += 32) d[k] = s[k];
    if (q == 0) cfw[1].h = cfw[0].h;
    __syncwarp();
}

struct SmallArgs {
    Ctx c;
    const int *sidx;   // [nm] stored (compact) index of magnetic cell i
    const int *snb;    // [6][nm] neighbour table (see SmallBuf)
    int nm;
};

// ONE: every worker owns at most one cell, whose state stays in registers (small_work_reg).
template <int NS, bool HU, bool ONE>
__global__ void __launch_bounds__(SMALL_NT, 1) small_kernel(SmallArgs A)
{
    extern __shared__ __align__(16) float sh[];
    __shared__ Local L;
    __shared__ Coef cfw[2];   // coefficients; feedback of the stages of parity 0 / 1
    __shared__ SmallRed R;
    __shared__ SmallPre pre;
    __shared__ int s_stop;
    constexpr int NQ = 3 * NS;
    const Ctx &c = A.c;
    const int nm = A.nm, tid = threadIdx.x;
    const bool ctl = tid < 32, helper = tid >= 32 && tid < SMALL_W0, worker = tid >= SMALL_W0;
    const size_t V = (size_t)NQ * nm;
    SmallBuf b;
    b.mb0 = sh;
    b.mb1 = sh + V;
    b.ms[0] = sh + 2 * V;
    b.ms[1] = sh + 3 * V;
    b.es = sh + 4 * V;
    b.kk = sh + 5 * V;
    b.uu = b.kk + 7 * V;
    int *nb = reinterpret_cast<int *>(sh + 12 * V + (HU ? (size_t)c.nmodes * nm : 0));
    b.nb = nb;
    if (tid == 0) {
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
        // fixed-point scale of the per-thread overlap partials (ceil(nm / workers) cells each)
        const int P = (nm + SMALL_WK - 1) / SMALL_WK;
        const float bound = 2.f * (float)(P > 1 ? P : 1) * fmaxf(c.umax, 1.f);
        const int k = SMALL_TBITS - (int)ceilf(log2f(bound));
        L.tscale = ldexpf(1.f, k);
        L.tshift = ilogb(c.red_scale) - k - 20;
        R.emax = 0u;
        R.bad = 0;
    }
    if (tid < 2 * 2 * MAXN) R.dig[tid / (2 * MAXN)][tid % (2 * MAXN)][0] =
                             R.dig[tid / (2 * MAXN)][tid % (2 * MAXN)][1] = 0;
    if (tid < 2 * c.nmodes) component_constants(c, tid, L);
    if (tid >= 32 && tid < 39) cfw[0].e[tid - 32] = cfw[1].e[tid - 32] = (float)dp_e(tid - 32);
    if (tid < c.nmodes) mode_constants(c, tid, L.mc + MC * tid);
    __syncthreads();
    {   // state, FSAL slope, profiles and neighbour table into shared memory
        const float *gm = L.mcur ? c.m[1] : c.m[0];
        float *mn = L.mcur ? b.mb1 : b.mb0;
        const float *gk1 = slope_buffer(c, L.kphys[0]);
        float *k1 = b.kk + L.kphys[0] * V;
        float *uu = b.kk + 7 * V;
        for (int i = tid; i < nm; i += SMALL_NT) {
            const int si = __ldg(A.sidx + i);
            if (!idx_ok(c, si, c.ncell, 15)) continue;
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                mn[q * nm + i] = gm[(size_t)q * c.ncell + si];
                k1[q * nm + i] = L.k1_valid ? gk1[(size_t)q * c.ncell + si] : 0.f;
            }
            if (HU)
                for (int n = 0; n < c.nmodes; n++)
                    uu[n * nm + i] = __ldg(c.u + (size_t)n * c.ncell + si);
#pragma unroll
            for (int d = 0; d < 6; d++) nb[d * nm + i] = __ldg(A.snb + d * nm + i);
        }
    }
    CellReg<NS> r;   // workers' cell in registers (ONE)
    if (ONE) {
        __syncthreads();
        const int i = tid - SMALL_W0;
        r.mcur = L.mcur;
        if (worker && i < nm) {
            const float *mn = L.mcur ? b.mb1 : b.mb0;
            const float *k1 = b.kk + L.kphys[0] * V;
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                r.mn[q] = mn[q * nm + i];
                r.k[0][q] = k1[q * nm + i];
            }
#pragma unroll
            for (int n = 0; n < MAXN; n++) r.u[n] = (HU && n < c.nmodes) ? b.uu[n * nm + i] : 1.f;
#pragma unroll
            for (int d = 0; d < 6; d++) {
                r.nbr[d] = nb[d * nm + i];
                if (r.nbr[d] >= 0 && !idx_ok(c, r.nbr[d], nm, 14)) r.nbr[d] = -1;
            }
        }
    }
    // Every thread passes the same sequence of block barriers (__syncthreads: attempt start,
    // end of stage 1, end of stage 7) and, per stage, one sums and one feedback barrier; the
    // loop conditions (s_stop, L.k1_valid) are read after a block barrier that follows their
    // last write.
    Cav7 cav7{0.0, 0.0, 0.f};
    for (;;) {
        if (ctl) {   // warp 0: the next attempt's size and its stage-2 set-up
            if (tid == 0) {
                s_stop = L.status != 0 || L.done;
                if (!s_stop) attempt_size(c, L);
            }
            __syncwarp();
            if (!s_stop && L.k1_valid) small_attempt_setup(L, cfw, c.nmodes);
        }
        __syncthreads();
        if (ONE && worker && L.mcur != r.mcur) {   // the last attempt was accepted: FSAL
            r.mcur = L.mcur;
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                r.mn[q] = r.m7[q];
                r.k[0][q] = r.k[6][q];
            }
        }
        if (s_stop) break;
        while (!L.k1_valid) {   // twice at an operator-split boundary (see controller<1>)
            if (ctl) {
                cavity_stage_value<1>(L, cfw[1], tid, tid < 2 * c.nmodes);
                small_control<1>(c, L, cfw, R);
                if (L.k1_valid) small_attempt_setup(L, cfw, c.nmodes);
            } else if (worker) {
                if (ONE) small_work_reg<NS, HU, 1>(c, nm, b, L, cfw[1], R, r);
                else small_work<NS, HU, 1>(c, nm, b, L, cfw[1], R);
            }
            __syncthreads();
        }
        if (ctl) {
            small_control_pre<2>(c, L, cfw, R, pre);
            small_control_pre<3>(c, L, cfw, R, pre);
            small_control_pre<4>(c, L, cfw, R, pre);
            small_control_pre<5>(c, L, cfw, R, pre);
            small_control_pre<6>(c, L, cfw, R, pre);
            // stage 7's cavity slope and cavity error norm while the workers run pass B
            const Team tm{0, 1, nullptr};
            cav7 = controller_cavity<7>(c, tm, L, cfw[1], small_control<7>(c, L, cfw, R));
            __syncwarp();
        } else if (helper) {   // the cavity terms of stages 2..6 known before their sums
            small_prepare<2>(c, L, pre);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                bar_sync_n(BAR_HELP, 64);
                if (k == 0) small_prepare<3>(c, L, pre);
                if (k == 1) small_prepare<4>(c, L, pre);
                if (k == 2) small_prepare<5>(c, L, pre);
                if (k == 3) small_prepare<6>(c, L, pre);
            }
        } else if (ONE) {
            const int i = tid - SMALL_W0;
            const float c21 = cfw[0].cf[1][0];
            if (i < nm) {
#pragma unroll
                for (int q = 0; q < NQ; q++) {
                    r.ms[q] = fmaf(c21, r.k[0][q], r.mn[q]);
                    b.ms[0][q * nm + i] = r.ms[q];
                }
            }
            small_work_reg<NS, HU, 2>(c, nm, b, L, cfw[0], R, r);
            small_work_reg<NS, HU, 3>(c, nm, b, L, cfw[1], R, r);
            small_work_reg<NS, HU, 4>(c, nm, b, L, cfw[0], R, r);
            small_work_reg<NS, HU, 5>(c, nm, b, L, cfw[1], R, r);
            small_work_reg<NS, HU, 6>(c, nm, b, L, cfw[0], R, r);
            small_work_reg<NS, HU, 7>(c, nm, b, L, cfw[1], R, r);
        } else {
            {   // m_2 = m_n + h a_21 k_1 of the worker's own cells
                const float *mn = L.mcur ? b.mb1 : b.mb0;
                const float *k1 = b.kk + L.kphys[0] * V;
                const float c21 = cfw[0].cf[1][0];
                for (int i = tid - SMALL_W0; i < nm; i += SMALL_WK)
#pragma unroll
                    for (int q = 0; q < NQ; q++)
                        b.ms[0][q * nm + i] = fmaf(c21, k1[q * nm + i], mn[q * nm + i]);
            }
            small_work<NS, HU, 2>(c, nm, b, L, cfw[0], R);
            small_work<NS, HU, 3>(c, nm, b, L, cfw[1], R);
            small_work<NS, HU, 4>(c, nm, b, L, cfw[0], R);
            small_work<NS, HU, 5>(c, nm, b, L, cfw[1], R);
            small_work<NS, HU, 6>(c, nm, b, L, cfw[0], R);
            small_work<NS, HU, 7>(c, nm, b, L, cfw[1], R);
        }
        __syncthreads();
        if (ctl) {   // accept decision: the workers' error maximum is complete
            const float emax = R.bad ? __int_as_float(0x7fffffff) : __uint_as_float(R.emax);
            __syncwarp();
            if (tid == 0) R.emax = 0u;
            const Team tm{0, 1, nullptr};
            controller_decide(c, tm, L, cav7, emax);
            __syncwarp();
        }
    }
    // write back: control block, state and FSAL slope
    if (tid == 0) store_local(c, L);
    {
        const float *mn = L.mcur ? b.mb1 : b.mb0;
        float *gm = L.mcur ? c.m[1] : c.m[0];
        const float *k1 = b.kk + L.kphys[0] * V;
        float *gk1 = const_cast<float *>(slope_buffer(c, L.kphys[0]));
        for (int i = tid; i < nm; i += SMALL_NT) {
            const int si = __ldg(A.sidx + i);
            if (!idx_ok(c, si, c.ncell, 16)) continue;
#pragma unroll
            for (int q = 0; q < NQ; q++) {
                gm[(size_t)q * c.ncell + si] = mn[q * nm + i];
                if (!ONE && L.k1_valid) gk1[(size_t)q * c.ncell + si] = k1[q * nm + i];
            }
        }
        if (ONE && worker && tid - SMALL_W0 < nm && L.k1_valid) {
            const int i = tid - SMALL_W0, si = __ldg(A.sidx + i);
            if (idx_ok(c, si, c.ncell, 16))
#pragma unroll
                for (int q = 0; q < NQ; q++) gk1[(size_t)q * c.ncell + si] = r.k[0][q];
        }
    }
}

template <int NS, bool HU>
static cudaError_t small_launch_variant(const SmallArgs &a, cudaStream_t s)
{
    auto *fn = a.nm <= SMALL_WK ? small_kernel<NS, HU, true> : small_kernel<NS, HU, false>;
    const size_t smem = small_smem_bytes(a.nm, NS, a.c.nmodes, HU);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<1, SMALL_NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_small(const Ctx &c, const int *sidx, const int *snb, int nm, cudaStream_t s)
{
    const SmallArgs a{c, sidx, snb, nm};
    if (c.nsub == 1) return c.u ? small_launch_variant<1, true>(a, s)
                                : small_launch_variant<1, false>(a, s);
    if (c.nsub == 2) return c.u ? small_launch_variant<2, true>(a, s)
                                : small_launch_variant<2, false>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace cmx
