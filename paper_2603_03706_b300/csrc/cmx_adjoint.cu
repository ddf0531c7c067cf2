// Reverse sweep of the discrete adjoint (sm_103a).
//
// For one checkpoint interval whose stage points were recorded by a replay, the persistent
// kernel walks the steps last to first and, inside a step, the Dormand-Prince stages 7 .. 2
// (and stage 1 on the run's first step).  With F_S the adjoint of stage point Y_S and
// w_S = h sum_{S'>S} a_{S'S} F_{S'} the adjoint of slope k_S (w_7 = adjoint of the FSAL slope
// that the next step received), one reverse stage computes, per magnetic cell,
//   Bbar  = pre [ w x m + alpha m x (m x w) ]                        (adjoint of the field)
//   F_S,m = pre [ B x w + alpha (w (m.B) + B (w.m) - 2 m (w.B)) ]     (torque, B held fixed)
//         + sum_nb w_d (Bbar_j - Bbar_i)                              (exchange stencil)
//         + anis (Bbar.k) k - dmg o sum_s Bbar_s - B_E Bbar_other      (anisotropy, demag, AFM)
//         + x: sum_n u_n mbar_re,n / (N_c nsub), y: -sum_n u_n mbar_im,n / (N_c nsub)  (overlaps)
// and the cell sums S_n = sum u_n Bbar_x (the feedback field's adjoint, Eq. (5), (13)) and
// w . dT/dalpha, reduced over the grid; the cavity part F_S,a and the parameter gradients follow
// in FP64 on every block's copy of the scalar state, as in the forward controller.  Stage 7
// adds the transpose of the renormalisation, J^T mbar = (mbar - n (n.mbar)) / |Y_7|; stage 2
// ends the step with mbar = sum_S F_S and k1bar = h sum_S a_{S1} F_S.
//
// The field adjoint depends only on the cell's own (m, w), so the stencil needs one halo cell:
// a 32 x 8 window marches through its columns plane by plane like the forward stage, holding
// (m, Bbar, presence) of four planes in shared memory; the global loads of plane p+2 are in
// flight while plane p is computed.
#include "cmx_stage.cuh"
#include "cmx_kernels.h"

namespace cmx {

template <int NS, int WX, int WY>
struct RevSmem {
    static constexpr int W = WX * WY, NQ = 3 * NS, R = 4;
    float mv[R][NQ][W];          // stage point m of four planes (0 where absent)
    float bb[R][NQ][W];          // field adjoint Bbar of four planes (0 where absent)
    float pr[R][W];              // presence
    int2 rows[8][WY];
    int2 rowc[ROWC][WY];         // row entries of the first ROWC planes of the stream
    int4 seg[MAX_BLOCK_SEGMENTS];
    int nseg;
    F2 red[32][MAXN + 1];
};

// Block copy of the scalar adjoint state (shared memory).
struct RevLocal {
    double Fa[7][2 * MAXN];      // cavity part of F_S (index S-1)
    double abar[2 * MAXN], k1a[2 * MAXN];
    double wa[2 * MAXN];         // cavity part of the slope adjoint w_S
    double as[2 * MAXN], mm[2 * MAXN];   // a_S and <m^->_S of the recorded forward
    double mc[MC * MAXN];        // mode constants (see MC)
    double gacc[NGRAD * MAXN];       // per mode: Re g~, Im g~, kappa, omega, Re gb~, Im gb~, K, Re P, Im P
    double galpha;
    double sums[MAXN + 1];
    double h, t0;                // step size and start time of the step
    double hA[7][6];             // h a_ij of the step (rows 1..6)
    double pc[3 * MAXN];         // per mode: pump Re P, Im P, frequency
    float cw[7], c1[7];          // h a_{S'S} and h a_{S'1} by S'-1
    float hrf[MAXN], ovr[MAXN], ovi[MAXN];
    unsigned bar_target;
};

// Raw operands of one window position of one plane, and what the centre computation keeps.
template <int NQ, int NWS>
struct RevRaw {
    float y[NQ], s[NWS][NQ];
    int idx;
    bool inner;
};

template <int NQ>
struct RevCen {
    float m[NQ], w[NQ], sf[NQ], k1[NQ], mb[NQ], u[MAXN];
    int idx;
};

__device__ __forceinline__ void red_add_release_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Parametric pump -i Q conj(a) = (qi ar - qr ai, -(qr ar + qi ai)), Q = P e^{-i wp t}, at time
// t: its (symmetric) Jacobian transposed onto the slope adjoint (wr, wi) -> out[0..1], and dL/dQ
// mapped to dL/d Re P, dL/d Im P -> out[2..3].  pp = (Re P, Im P, wp).  Out of line, so that the
// FP64 sine and cosine do not weigh on the reverse stage when no pump is set.
static __device__ __noinline__ void pump_adjoint(const double *pp, double t, double ar, double ai,
                                                 double wr, double wi, double *out)
{
    double sn, cs;
    sincos(pp[2] * t, &sn, &cs);
    const double qr = pp[0] * cs + pp[1] * sn, qi = pp[1] * cs - pp[0] * sn;
    out[0] = qi * wr - qr * wi;
    out[1] = -(qr * wr + qi * wi);
    const double lqr = -ai * wr - ar * wi, lqi = ar * wr - ai * wi;
    out[2] = lqr * cs - lqi * sn;
    out[3] = lqr * sn + lqi * cs;
}

// Barrier of all blocks of the launch (monotonic arrival counter, bounded wait; on time-out the
// status becomes CMX_ETIMEOUT and every block leaves).
__device__ bool rev_barrier(const AdjArgs &A, RevLocal &L, int where)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        L.bar_target += gridDim.x;
        red_add_release_u32(&A.ctl->bar_count, 1u);
        const unsigned long long t0 = global_timer_ns();
        unsigned spins = 0;
        while ((int)(ld_acquire(&A.ctl->bar_count) - L.bar_target) < 0) {
            if ((++spins & 31u) == 0) {
                if (ld_volatile_int(&A.ctl->status) != 0) {
                    s_ok = 0;
                    break;
                }
                if (global_timer_ns() - t0 > (unsigned long long)A.f.timeout_ns) {
                    atomicCAS(&A.ctl->status, 0, (int)CMX_ETIMEOUT);
                    A.ctl->timeout_where = where;
                    s_ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return s_ok > 0;
}

// Block sums (compensated pairs, fixed shuffle order) of the per-thread partials into the
// block's slot of A.part, then, after the barrier, the fixed-order grid sum by every block.
template <int NT>
__device__ void rev_block_reduce(const AdjArgs &A, F2 (*red)[MAXN + 1], const float *acc, int nq)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q <= MAXN; q++) {
        if (q >= nq) break;
        // modes 0..nq-2 in acc[q], the alpha sum (last) in acc[MAXN]
        F2 v = {q == nq - 1 ? acc[MAXN] : acc[q], 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = f2_add(v, f2_shfl_xor(v, o));
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        F2 s = {0.f, 0.f};
        for (int w = 0; w < NT / 32; w++) s = f2_add(s, red[w][threadIdx.x]);
        A.part[(size_t)blockIdx.x * nq + threadIdx.x] = make_float2(s.hi, s.lo);
    }
}

template <int NT>
__device__ void rev_grid_reduce(const AdjArgs &A, F2 (*red)[MAXN + 1], double *out, int nq)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
    int QP = 1;
    while (QP < nq) QP <<= 1;
    const int q = threadIdx.x & (QP - 1), grp = threadIdx.x / QP, ngrp = NT / QP;
    F2 s = {0.f, 0.f};
    if (q < nq) {
        // all of this thread's partials in one round of loads, then the fixed-order sum
        constexpr int KMAX = 8;
        float2 v[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; k++) {
            const int b = grp + k * ngrp;
            v[k] = b < G ? __ldcg(A.part + (size_t)b * nq + q) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < KMAX; k++) s = f2_add(s, {v[k].x, v[k].y});
        for (int b = grp + KMAX * ngrp; b < G; b += ngrp) {
            const float2 w = __ldcg(A.part + (size_t)b * nq + q);
            s = f2_add(s, {w.x, w.y});
        }
    }
    for (int o = 16; o >= QP; o >>= 1) s = f2_add(s, f2_shfl_xor(s, o));
    __syncthreads();   // red[] of the block reduction may still be read
    if (lane < QP && lane < nq) red[warp][lane] = s;
    __syncthreads();
    if (threadIdx.x < nq) {
        F2 v = {0.f, 0.f};
        for (int w = 0; w < NT / 32; w++) v = f2_add(v, red[w][threadIdx.x]);
        out[threadIdx.x] = (double)v.hi + (double)v.lo;
    }
    __syncthreads();
}

// Number of arrays combined into the slope adjoint at stage S: the FSAL slope's adjoint at
// stages 7 and 1, the stage-point adjoints F_{S+1..7} otherwise.
__host__ __device__ constexpr int rev_nsrc(int S) { return (S == 1 || S == 7) ? 1 : 7 - S; }

// Centre cell of plane p: F_S for this cell, the partial sums, dL/du, the outputs.
template <int NS, int WX, int WY, bool HU, int S>
__device__ __forceinline__ void rev_cell(const AdjArgs &A, RevSmem<NS, WX, WY> &sm,
                                         const RevLocal &L, const RevCen<3 * NS> &ce, int p,
                                         float *acc)
{
    using SM = RevSmem<NS, WX, WY>;
    constexpr int R = SM::R;
    const Ctx &c = A.f;
    const int i = threadIdx.x, idx = ce.idx;
    if (idx < 0) return;
    const size_t nc = (size_t)c.ncell;
    const int sp = (p + R - 1) % R, sc = p % R, sn = (p + 1) % R;
    const float nx_ = sm.pr[sc][i - 1] + sm.pr[sc][i + 1];
    const float ny_ = sm.pr[sc][i - WX] + sm.pr[sc][i + WX];
    const float nz_ = sm.pr[sp][i] + sm.pr[sn][i];

    float B[NS][3], Gx[NS][3], bc[NS][3];
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = s * 3 + k;
            const float cm = ce.m[q];
            B[s][k] = c.wx * (sm.mv[sc][q][i - 1] + sm.mv[sc][q][i + 1] - nx_ * cm) +
                      c.wy * (sm.mv[sc][q][i - WX] + sm.mv[sc][q][i + WX] - ny_ * cm) +
                      c.wz * (sm.mv[sp][q][i] + sm.mv[sn][q][i] - nz_ * cm);
            const float cb = sm.bb[sc][q][i];
            bc[s][k] = cb;
            Gx[s][k] = c.wx * (sm.bb[sc][q][i - 1] + sm.bb[sc][q][i + 1] - nx_ * cb) +
                       c.wy * (sm.bb[sc][q][i - WX] + sm.bb[sc][q][i + WX] - ny_ * cb) +
                       c.wz * (sm.bb[sp][q][i] + sm.bb[sn][q][i] - nz_ * cb);
        }
    float mt[3], bt[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        mt[k] = NS == 2 ? ce.m[k] + ce.m[3 + k] : ce.m[k];
        bt[k] = NS == 2 ? bc[0][k] + bc[1][k] : bc[0][k];
    }
    float brf = 0.f, ovx = 0.f, ovy = 0.f;
#pragma unroll
    for (int n = 0; n < MAXN; n++)
        if (n < c.nmodes) {
            const float un = HU ? ce.u[n] : 1.f;
            brf = fmaf(un, L.hrf[n], brf);
            ovx = fmaf(un, L.ovr[n], ovx);
            ovy = fmaf(un, L.ovi[n], ovy);
        }
    const float ca = -2.f * c.alpha / (1.f + c.alpha * c.alpha);
    float F[NS][3];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const float *m = ce.m + 3 * s, *w = ce.w + 3 * s;
        const float mk = m[0] * c.ku[0] + m[1] * c.ku[1] + m[2] * c.ku[2];
        float b[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float v = B[s][k] + c.anis * mk * c.ku[k] + c.B0[k] - c.dmg[k] * mt[k];
            if (NS == 2) v -= c.BE * ce.m[3 * (1 - s) + k];
            b[k] = v;
        }
        b[0] += brf;
        const float t1[3] = {m[1] * b[2] - m[2] * b[1], m[2] * b[0] - m[0] * b[2],
                             m[0] * b[1] - m[1] * b[0]};
        const float t2[3] = {m[1] * t1[2] - m[2] * t1[1], m[2] * t1[0] - m[0] * t1[2],
                             m[0] * t1[1] - m[1] * t1[0]};
        const float mB = m[0] * b[0] + m[1] * b[1] + m[2] * b[2];
        const float wm = w[0] * m[0] + w[1] * m[1] + w[2] * m[2];
        const float wB = w[0] * b[0] + w[1] * b[1] + w[2] * b[2];
        const float bxw[3] = {b[1] * w[2] - b[2] * w[1], b[2] * w[0] - b[0] * w[2],
                              b[0] * w[1] - b[1] * w[0]};
        const float bk = bc[s][0] * c.ku[0] + bc[s][1] * c.ku[1] + bc[s][2] * c.ku[2];
        float da = 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float f = c.pre * (bxw[k] + c.alpha * (w[k] * mB + b[k] * wm - 2.f * m[k] * wB));
            f += Gx[s][k] + c.anis * bk * c.ku[k] - c.dmg[k] * bt[k];
            if (NS == 2) f -= c.BE * bc[1 - s][k];
            F[s][k] = f;
            // w . dT/dalpha, T = pre (t1 + alpha t2), d pre/d alpha = pre ca
            da = fmaf(w[k], c.pre * (ca * (t1[k] + c.alpha * t2[k]) + t2[k]), da);
        }
        F[s][0] += ovx;
        F[s][1] += ovy;
        if (S == 7) {   // transpose of the renormalisation m_{n+1} = Y_7 / |Y_7|
            const float *mb = ce.mb + 3 * s;
            const float r = rsqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            const float nl = (m[0] * mb[0] + m[1] * mb[1] + m[2] * mb[2]) * r;
#pragma unroll
            for (int k = 0; k < 3; k++) F[s][k] += (mb[k] - m[k] * r * nl) * r;
        }
        acc[MAXN] += da;
    }
    // feedback field adjoint and dL/du
    const float bx = bt[0];
#pragma unroll
    for (int n = 0; n < MAXN; n++)
        if (n < c.nmodes) {
            const float un = HU ? ce.u[n] : 1.f;
            acc[n] = fmaf(un, bx, acc[n]);
            if (HU && A.ubar) {
                float *ub = A.ubar + (size_t)n * nc + idx;
                // fire-and-forget reduction: the cell's accumulator belongs to this thread in
                // every stage, so the additions keep their order, and no load waits here
                atomicAdd(ub, L.hrf[n] * bx + L.ovr[n] * mt[0] + L.ovi[n] * mt[1]);
            }
        }
    // outputs
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = s * 3 + k;
            const size_t o = (size_t)q * nc + idx;
            if (S >= 3) {
                A.F[S >= 3 ? S - 3 : 0][o] = F[s][k];
            } else if (S == 2) {
                A.mbar[o] = F[s][k] + ce.sf[q];
                A.k1bar[o] = fmaf(L.c1[1], F[s][k], ce.k1[q]);
            } else {
                A.mbar[o] = ce.mb[q] + F[s][k];
            }
        }
}

// One reverse stage over the block's columns.
template <int NS, int WX, int WY, bool HU, int S>
__device__ void rev_tiles(const AdjArgs &A, RevSmem<NS, WX, WY> &sm, const RevLocal &L, int jj,
                          float *acc)
{
    using SM = RevSmem<NS, WX, WY>;
    constexpr int NQ = SM::NQ, R = SM::R, NWS = rev_nsrc(S), AHEAD = 4;
    constexpr bool MB = (S == 1 || S == 7);
    const Ctx &c = A.f;
    __syncthreads();   // the previous stage may still read the rings
    if (sm.nseg == 0) return;
    const size_t nc = (size_t)c.ncell;
    int gend = 0;
    for (int t = 0; t < sm.nseg; t++) gend += sm.seg[t].w - sm.seg[t].z + 2;
    const int i = threadIdx.x, r = i / WX, col = i - (i / WX) * WX;
    const bool corner = (r == 0 || r == WY - 1) && (col == 0 || col == WX - 1);
    const bool inner_pos = r >= 1 && r <= WY - 2 && col >= 1 && col <= WX - 2;
    const float *Y = (S == 1) ? A.m_first
                              : A.rec_m + ((size_t)jj * 6 + (S >= 2 ? S - 2 : 0)) * NQ * nc;
    const float *src[NWS];
    float cwv[NWS], c1v[NWS];
#pragma unroll
    for (int a = 0; a < NWS; a++) {
        if (S == 1 || S == 7) {
            src[a] = A.k1bar;
            cwv[a] = 1.f;
            c1v[a] = 0.f;
        } else {
            const int t = S + 1 + a;   // source stage S' = t
            src[a] = A.F[t - 3];
            cwv[a] = L.cw[t - 1];
            c1v[a] = L.c1[t - 1];
        }
    }
    Cursor crow = cursor_start(sm), cis = crow;
    auto load_rows = [&](int g) {
        if (i < WY && g < gend) {
            cursor_seek(sm, crow, g);
            sm.rows[g & 7][i] = g < ROWC ? sm.rowc[g][i]
                                         : row_entry(c, crow.y0 - 1 + i, crow.z0 - 1 + (g - crow.off));
        }
    };
    auto issue = [&](int g, RevRaw<NQ, NWS> &rw) {
        rw.idx = -1;
        rw.inner = false;
        if (g >= gend) return;
        cursor_seek(sm, cis, g);
        const int q = g - cis.off;
        rw.inner = inner_pos && q >= 1 && q <= cis.np - 2;
        const int idx = corner ? -1 : row_index(c, sm.rows[g & 7][r], cis.x0 - 1 + col);
        rw.idx = idx;
        if (idx < 0) return;
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            rw.y[k] = __ldg(Y + (size_t)k * nc + idx);
#pragma unroll
            for (int a = 0; a < NWS; a++) rw.s[a][k] = __ldcg(src[a] + (size_t)k * nc + idx);
        }
    };
    auto write = [&](int g, const RevRaw<NQ, NWS> &rw, RevCen<NQ> &ce) {
        const int vs = g % R;
        const bool here = rw.idx >= 0;
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            float w = 0.f, sf = 0.f, k1 = 0.f;
            if (here)
#pragma unroll
                for (int a = 0; a < NWS; a++) {
                    w = fmaf(cwv[a], rw.s[a][k], w);
                    if (S == 2) {
                        sf += rw.s[a][k];
                        k1 = fmaf(c1v[a], rw.s[a][k], k1);
                    }
                }
            ce.m[k] = here ? rw.y[k] : 0.f;
            ce.w[k] = w;
            ce.sf[k] = sf;
            ce.k1[k] = k1;
        }
        // centre-only operands, loaded one plane before their use
        const bool cen_here = here && rw.inner;
#pragma unroll
        for (int k = 0; k < NQ; k++)
            ce.mb[k] = (MB && cen_here) ? __ldcg(A.mbar + (size_t)k * nc + rw.idx) : 0.f;
#pragma unroll
        for (int n = 0; n < MAXN; n++)
            ce.u[n] = (HU && cen_here && n < c.nmodes) ? __ldg(c.u + (size_t)n * nc + rw.idx) : 1.f;
#pragma unroll
        for (int s = 0; s < NS; s++) {
            const float *m = ce.m + 3 * s, *w = ce.w + 3 * s;
            // Bbar = pre (w x m + alpha m x (m x w))
            const float wxm[3] = {w[1] * m[2] - w[2] * m[1], w[2] * m[0] - w[0] * m[2],
                                  w[0] * m[1] - w[1] * m[0]};
            const float mxw[3] = {-wxm[0], -wxm[1], -wxm[2]};
            const float mmw[3] = {m[1] * mxw[2] - m[2] * mxw[1], m[2] * mxw[0] - m[0] * mxw[2],
                                  m[0] * mxw[1] - m[1] * mxw[0]};
#pragma unroll
            for (int k = 0; k < 3; k++) {
                sm.mv[vs][s * 3 + k][i] = m[k];
                sm.bb[vs][s * 3 + k][i] = c.pre * fmaf(c.alpha, mmw[k], wxm[k]);
            }
        }
        sm.pr[vs][i] = here ? 1.f : 0.f;
        ce.idx = (here && rw.inner) ? rw.idx : -1;
    };
    for (int g = 0; g <= AHEAD; g++) load_rows(g);
    __syncthreads();
    RevRaw<NQ, NWS> nx;
    RevCen<NQ> cen, cnx;
    issue(0, nx);
    write(0, nx, cen);
    if (gend > 1) {
        issue(1, nx);
        write(1, nx, cen);
    }
    issue(2, nx);
    for (int p = 1; p <= gend - 2; p++) {
        load_rows(p + AHEAD);
        write(p + 1, nx, cnx);
        __syncthreads();
        issue(p + 2, nx);
        rev_cell<NS, WX, WY, HU, S>(A, sm, L, cen, p, acc);
        cen = cnx;
    }
}

// Reverse stage S of interval step jj: scalar prelude, cell sweep, grid sums, cavity adjoint and
// parameter gradients.  Returns false if the run must stop.
template <int NS, int WX, int WY, bool HU, int S>
__device__ bool rev_stage(const AdjArgs &A, RevSmem<NS, WX, WY> &sm, RevLocal &L, int jj)
{
    const Ctx &c = A.f;
    const int tid = threadIdx.x, N = c.nmodes;
    if (tid < 2 * N) {
        const double *ra = (S == 1) ? A.a_first : A.rec_a + ((size_t)jj * 7 + (S - 1)) * 4 * N;
        L.as[tid] = ra[tid];
        L.mm[tid] = (S == 1) ? ra[4 * N + tid] : ra[2 * N + tid];
        double w = 0.0;
        if (S == 1 || S == 7) {
            w = L.k1a[tid];
        } else {
#pragma unroll
            for (int t = S + 1; t <= 7; t++)
                if (dp_a(t - 1, S - 1) != 0.0) w += L.hA[t - 1][S - 1] * L.Fa[t - 1][tid];
        }
        L.wa[tid] = w;
    }
    if (tid >= 32 && tid < 39) {
        const int t = tid - 32;   // S' - 1
        L.cw[t] = (S != 1 && S != 7 && t + 1 > S) ? (float)(L.h * dp_a(t, S - 1)) : 0.f;
        L.c1[t] = (float)(L.h * dp_a(t, 0));
    }
    // FP64 scalar work is spread over warps: a warp holds an FP64 instruction for about 64
    // cycles, while several warps of an SM run them at once
    if (tid >= 64 && tid < 64 + N) {   // feedback coefficient of mode n at a_S (Eq. (5), (13))
        const int n = tid - 64;
        const double *ra = (S == 1) ? A.a_first : A.rec_a + ((size_t)jj * 7 + (S - 1)) * 4 * N;
        const double *q = L.mc + MC * n;
        L.hrf[n] = (float)(c.two_over_gamma * (q[4] * ra[2 * n] - q[5] * ra[2 * n + 1]));
    }
    __syncthreads();
    if (tid < N) {
        const double *q = L.mc + MC * tid;
        const double gr = q[2], gi = q[3];
        const double wr = L.wa[2 * tid], wi = L.wa[2 * tid + 1];
        // adjoint of <m^->_n from da/dt = ... + i g~ <m^->
        const double mbr = -gi * wr + gr * wi;
        const double sc = c.inv_nmag / NS;
        L.ovr[tid] = (float)(sc * mbr);
    }
    if (tid >= 96 && tid < 96 + N) {   // its imaginary part on warp 3
        const int n = tid - 96;
        const double *q = L.mc + MC * n;
        const double gr = q[2], gi = q[3];
        const double wr = L.wa[2 * n], wi = L.wa[2 * n + 1];
        const double mbi = -gr * wr - gi * wi;
        const double sc = c.inv_nmag / NS;
        L.ovi[n] = (float)(-sc * mbi);
    }
    __syncthreads();
    float acc[MAXN + 1];
#pragma unroll
    for (int q = 0; q <= MAXN; q++) acc[q] = 0.f;
    rev_tiles<NS, WX, WY, HU, S>(A, sm, L, jj, acc);
    rev_block_reduce<WX * WY>(A, sm.red, acc, N + 1);
    if (!rev_barrier(A, L, S)) return false;
    rev_grid_reduce<WX * WY>(A, sm.red, L.sums, N + 1);
    if (tid < N) {
        const int n = tid;
        const double Sn = L.sums[n], tg = c.two_over_gamma;
        const double *q = L.mc + MC * n;
        const double w = q[0], k = q[1], gbr = q[4], gbi = q[5], K = q[6];
        const double wr = L.wa[2 * n], wi = L.wa[2 * n + 1];
        const double ar = L.as[2 * n], ai = L.as[2 * n + 1];
        // feedback field adjoint through gb~ (the backward coupling), then the cavity equation
        double fr = -k * wr - w * wi + tg * gbr * Sn;
        double fi = w * wr - k * wi - tg * gbi * Sn;
        // self-Kerr -i K |a|^2 a = (K |a|^2 ai, -K |a|^2 ar); its Jacobian terms vanish at K = 0,
        // and FP64 instructions are expensive on this part of the stage
        if (K != 0.0) {
            fr += wr * 2.0 * K * ar * ai - wi * K * (3.0 * ar * ar + ai * ai);
            fi += wr * K * (ar * ar + 3.0 * ai * ai) - wi * 2.0 * K * ar * ai;
        }
        if (c.has_pump) {
            const double ts = S == 1 ? L.t0 : L.t0 + dp_c(S - 1) * L.h;
            double o[4];
            pump_adjoint(L.pc + 3 * n, ts, ar, ai, wr, wi, o);
            fr += o[0];
            fi += o[1];
            L.gacc[NGRAD * n + 7] += o[2];
            L.gacc[NGRAD * n + 8] += o[3];
        }
        if (S == 7) {
            fr += L.abar[2 * n];
            fi += L.abar[2 * n + 1];
        }
        L.Fa[S - 1][2 * n] = fr;
        L.Fa[S - 1][2 * n + 1] = fi;
    }
    // the gradient sums of the stage, beside warp 0's cavity adjoint: g~ (and gb~) on warp 1,
    // kappa and omega on warp 2, K on warp 3
    if ((tid >= 32 && tid < 32 + N) || (tid >= 64 && tid < 64 + N) || (tid >= 96 && tid < 96 + N)) {
        const int n = tid & 31;
        const double Sn = L.sums[n], tg = c.two_over_gamma;
        const double wr = L.wa[2 * n], wi = L.wa[2 * n + 1];
        const double ar = L.as[2 * n], ai = L.as[2 * n + 1];
        if (tid < 64) {
            const double mr = L.mm[2 * n], mi = L.mm[2 * n + 1];
            const int fb = c.has_gb ? 4 : 0;   // feedback gradients: gb~ if separate, else g~
            L.gacc[NGRAD * n + 0] += -mi * wr + mr * wi;
            L.gacc[NGRAD * n + 1] += -mr * wr - mi * wi;
            L.gacc[NGRAD * n + fb] += tg * ar * Sn;
            L.gacc[NGRAD * n + fb + 1] -= tg * ai * Sn;
        } else if (tid < 96) {
            L.gacc[NGRAD * n + 2] += -ar * wr - ai * wi;
            L.gacc[NGRAD * n + 3] += ai * wr - ar * wi;
        } else {
            const double s2 = ar * ar + ai * ai;
            L.gacc[NGRAD * n + 6] += s2 * (wr * ai - wi * ar);
        }
    }
    if (tid == 32 + MAXN) L.galpha += L.sums[N];
    __syncthreads();
    if (S == 2 && tid < 2 * N) {
        double sy = 0.0;
#pragma unroll
        for (int s = 2; s <= 7; s++) sy += L.Fa[s - 1][tid];
        if (A.dL_da) sy += A.dL_da[(size_t)(A.step0 + jj) * 2 * N + tid];
        L.abar[tid] = sy;
    }
    if (S == 2 && tid >= 32 && tid < 32 + 2 * N) {   // warp 1, beside the sum above
        const int q = tid - 32;
        double sk = 0.0;
#pragma unroll
        for (int s = 2; s <= 7; s++) sk += L.hA[s - 1][0] * L.Fa[s - 1][q];
        L.k1a[q] = sk;
    }
    if (S == 1 && tid < 2 * N) L.abar[tid] += L.Fa[0][tid];
    __syncthreads();
    return true;
}

// One sublattice: two 256-thread blocks per SM (128 registers; the more resident warps hide the
// per-plane latency better than the registers they cost); two sublattices: one block.
template <int NS, int WX, int WY, bool HU>
__global__ void __launch_bounds__(WX *WY, NS == 1 ? 2 : 1) rev_kernel(AdjArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<RevSmem<NS, WX, WY> *>(smem_raw);
    __shared__ RevLocal L;
    const Ctx &c = A.f;
    const int tid = threadIdx.x, N = c.nmodes;
    {
        const int sb = __ldg(&c.seg_begin[blockIdx.x]), se = __ldg(&c.seg_begin[blockIdx.x + 1]);
        if (tid == 0) sm.nseg = se - sb;
        for (int t = tid; t < se - sb; t += WX * WY) sm.seg[t] = __ldg(&c.tiles[sb + t]);
    }
    if (tid < 2 * N) {
        L.abar[tid] = A.ctl->abar[tid];
        L.k1a[tid] = A.ctl->k1a[tid];
    }
    if (tid < NGRAD * N) L.gacc[tid] = 0.0;
    if (tid < N) {
        mode_constants(c, tid, L.mc + MC * tid);
        double pr = c.pump_re[0], pi = c.pump_im[0], pw = c.pump_w[0];
#pragma unroll
        for (int u = 1; u < MAXN; u++)
            if (tid == u) {
                pr = c.pump_re[u];
                pi = c.pump_im[u];
                pw = c.pump_w[u];
            }
        L.pc[3 * tid] = pr;
        L.pc[3 * tid + 1] = pi;
        L.pc[3 * tid + 2] = pw;
    }
    if (tid == 0) {
        L.galpha = 0.0;
        L.bar_target = 0;
    }
    __syncthreads();
    if (sm.nseg > 0) {   // row entries of the first planes of the stream, once per launch
        int gend = 0;
        for (int t = 0; t < sm.nseg; t++) gend += sm.seg[t].w - sm.seg[t].z + 2;
        const int n = (gend < ROWC ? gend : ROWC) * WY;
        for (int e = tid; e < n; e += WX * WY) {
            const int g = e / WY, r = e - g * WY;
            Cursor cu = cursor_start(sm);
            cursor_seek(sm, cu, g);
            sm.rowc[g][r] = row_entry(c, cu.y0 - 1 + r, cu.z0 - 1 + (g - cu.off));
        }
    }
    __syncthreads();
    bool ok = true;
    for (int jj = A.nsteps - 1; jj >= 0 && ok; jj--) {
        if (tid == 0) {
            L.h = A.dts[jj];
            L.t0 = A.rec_t ? A.rec_t[jj] : 0.0;
        }
        if (tid >= 32 && tid < 32 + 36) {   // the step's weights h a_ij, once for its six stages
            const int q = tid - 32;
            double a = 0.0;
#pragma unroll
            for (int i = 1; i < 7; i++)
#pragma unroll
                for (int j = 0; j < 6; j++)
                    if (q == (i - 1) * 6 + j) a = dp_a(i, j);
            L.hA[1 + q / 6][q % 6] = A.dts[jj] * a;
        }
        __syncthreads();
        ok = rev_stage<NS, WX, WY, HU, 7>(A, sm, L, jj) && rev_stage<NS, WX, WY, HU, 6>(A, sm, L, jj) &&
             rev_stage<NS, WX, WY, HU, 5>(A, sm, L, jj) && rev_stage<NS, WX, WY, HU, 4>(A, sm, L, jj) &&
             rev_stage<NS, WX, WY, HU, 3>(A, sm, L, jj) && rev_stage<NS, WX, WY, HU, 2>(A, sm, L, jj);
        if (ok && A.step0 + jj == 0) ok = rev_stage<NS, WX, WY, HU, 1>(A, sm, L, jj);
    }
    if (ok && blockIdx.x == 0) {
        if (tid < 2 * N) {
            A.ctl->abar[tid] = L.abar[tid];
            A.ctl->k1a[tid] = L.k1a[tid];
        }
        if (tid < NGRAD * N) A.ctl->gacc[tid] += L.gacc[tid];
        if (tid == 0) A.ctl->galpha += L.galpha;
    }
}

// ---------------------------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------------------------
template <int NS, bool HU>
static cudaError_t rev_launch_variant(const AdjArgs &a, int blocks, cudaStream_t s)
{
    auto *fn = rev_kernel<NS, REV_WX, REV_WY, HU>;
    const size_t smem = sizeof(RevSmem<NS, REV_WX, REV_WY>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    AdjArgs aa = a;
    void *args[] = {&aa};
    return cudaLaunchCooperativeKernel((const void *)fn, dim3(blocks), dim3(REV_WX * REV_WY),
                                       args, smem, s);
}

template <int NS, bool HU>
static int rev_occupancy()
{
    auto *fn = rev_kernel<NS, REV_WX, REV_WY, HU>;
    const size_t smem = sizeof(RevSmem<NS, REV_WX, REV_WY>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, REV_WX * REV_WY, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_reverse(const AdjArgs &a, int blocks, cudaStream_t s)
{
    const bool hu = a.f.u != nullptr;
    if (a.f.nsub == 1) return hu ? rev_launch_variant<1, true>(a, blocks, s)
                                 : rev_launch_variant<1, false>(a, blocks, s);
    if (a.f.nsub == 2) return hu ? rev_launch_variant<2, true>(a, blocks, s)
                                 : rev_launch_variant<2, false>(a, blocks, s);
    return cudaErrorInvalidValue;
}

int reverse_blocks_per_sm(int nsub, bool has_u)
{
    if (nsub == 1) return has_u ? rev_occupancy<1, true>() : rev_occupancy<1, false>();
    if (nsub == 2) return has_u ? rev_occupancy<2, true>() : rev_occupancy<2, false>();
    return 0;
}

}  // namespace cmx
