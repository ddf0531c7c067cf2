// Stage code of the dense-box path (sm_103a): grids whose rows are magnetic over the whole box
// (films and full boxes: no mask), stored as dense (nz, ny, nxs) arrays per component, nxs = nx
// rounded up to a multiple of 8.  The stage arithmetic is that of cmx_stage.cuh (field, slope,
// stored next stage value, error partial, renormalised new state, overlap partials; each combine
// the same FMA chain); what differs is how a plane reaches shared memory and how presence is
// known:
//   - the copies of a plane are tensor copies (cp.async.bulk.tensor) that one thread issues, a
//     few per plane, with completion counted in bytes on an mbarrier, instead of one 4-byte
//     cp.async per thread, array and component with its own address arithmetic;
//   - a cell's presence and its neighbour counts follow from its coordinates, and positions
//     outside the box read as the copies' zero fill (an absent neighbour contributes 0).
//
// Per plane z of a block's stream, for the tile x0 .. x0+31, y0 .. y0+WY-1:
//   tile box  stage values at x0-4 .. x0+35, y0-1 .. y0+WY, every component (the copy's start
//             must lie on 16 bytes, hence x0-4); stage 2 also the slope k1 over the same box;
//   operands  the combine's operand arrays over the tile's own cells (32 x WY, every
//             component) and, with mode profiles, the profiles there.
// A ring of RING tile slots (planes p-1, p, p+1 read by the stencil of plane p, plane p+2 in
// flight) and D operand slots, one mbarrier each, initialised at the start of every stage.
// Iteration p waits for plane p+1's tile (at stage 2 it forms the tile's values m_n + h a_21 k_1
// in place), publishes it with the block barrier, lets lane 0 of warps 1 .. NW-1 issue plane
// p+2's tile and plane p+1's operands (dealt round-robin) into the slots that the barrier has
// just freed, and computes plane p, waiting for its operands where they are first used.  The
// copies at a stage's start are issued by one producer thread outside warp 0.  Halo planes
// (the first and last plane of a segment) get a tile and no operands: their operand phase is
// completed by a plain arrival.  (Measured and not kept: releasing slots per warp on a second
// mbarrier instead of the block barrier, 3 % slower; L2 prefetches of the boxes two planes
// ahead of their copies, 20 % slower.)
#pragma once

#include <cuda.h>

#include "cmx_stage.cuh"

namespace cmx {

constexpr int DX = 40;     // tile box width in cells
constexpr int DOFF = 4;    // box column of the tile's x0

// Tensor maps of a dense problem (device memory, one CUtensorMap each, 128-byte aligned): the
// tile box (DX x (WY+2) x 1 x nq) of m[0], m[1], msv[0], msv[1] and the seven slope buffers; the
// operand box (32 x WY x 1 x nq) of m[0], m[1], the slope buffers and es; the profiles' box
// (32 x WY x 1 x nmodes).
enum : int {
    TMT_M = 0,     // + 0 / 1
    TMT_MSV = 2,   // + 0 / 1
    TMT_K = 4,     // + physical slope buffer 0..6
    TMO_M = 11,    // + 0 / 1
    TMO_K = 13,    // + physical slope buffer 0..6
    TMO_ES = 20,
    TMO_U = 21,
    TM_COUNT = 22
};

// The tensor maps of a dense launch, built on the host from the launch's own buffers and passed
// by value (kernel parameter space).
struct DenseMaps {
    CUtensorMap map[TM_COUNT];
};

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory before later tensor copies
// (async proxy) into it.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's generic-proxy global stores (stage values, slopes, state written during a
// stage) before tensor copies that read them: the writers fence before the stage's grid
// barrier, the issuing thread again after it, before its first copy of the next stage.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the completion of the barrier's phase of the given parity, bounded by c.timeout_ns:
// on time-out the run's status becomes CMX_ETIMEOUT (site `where`) and false is returned (the
// engine stops at the stage's grid barrier).
__device__ __forceinline__ bool mbar_wait(const Ctx &c, unsigned long long *bar, unsigned parity,
                                          int where)
{
    const unsigned a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned spins = 0;; spins++) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if (spins == 0) {
            t0 = global_timer_ns();
        } else if ((spins & 63u) == 0 && global_timer_ns() - t0 > (unsigned long long)c.timeout_ns) {
            if (atomicCAS(&c.ctl->status, 0, (int)CMX_ETIMEOUT) == 0) c.ctl->timeout_where = where;
            return false;
        }
    }
}

// Tensor copy of the box at (x, y, z, 0) of tensor map `map` into shared memory at dst,
// completing `bytes` on bar (the caller announces them with mbar_arrive_expect_tx).
__device__ __forceinline__ void tma_load4(void *dst, const void *map, int x, int y, int z,
                                          unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
                 "l"(map), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(bar))
                 : "memory");
}

// The same with an L2 eviction-priority policy (streamed operands: evict_first).
__device__ __forceinline__ void tma_load4_hint(void *dst, const void *map, int x, int y, int z,
                                               unsigned long long *bar, unsigned long long pol)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 ".L2::cache_hint [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(smem_u32(dst)),
                 "l"(map), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(bar)), "l"(pol)
                 : "memory");
}

// Shared memory of a dense-path block of 32 x WY threads (one cell each).
template <int NS, int WY, bool HU>
struct DenseSmem {
    static constexpr int NQ = NS * 3;
    static constexpr int NT = 32 * WY, CW = 32 * WY;
    static constexpr int PY = WY + 2, P = DX * PY;            // tile box positions per component
    static constexpr int TSLOT = (NQ * P + 31) / 32 * 32;     // floats per ring slot
    static constexpr int NAMAX = 5;                           // m_n + at most four slopes
    static constexpr int D = 2;                               // operand slots
    static constexpr int RING = D + 2;                        // tile slots
    static constexpr int OPSLOT = NAMAX * NQ * CW;
    static constexpr int SIDE = 2 * NQ * CW;                  // stage 2: k1 box after 2 operands
    static constexpr int USLOT = HU ? MAXN * CW : 32;
    // the thread that initialises the barriers and issues the copies: lane 0 of the last warp,
    // so that warp 0, which runs the controller's warp-synchronous shuffles right after a
    // stage's first copies are issued, never diverges around the issue
    static constexpr int PROD = NT - 32;
    static_assert(SIDE + NQ * P <= OPSLOT, "stage-2 side buffer");
    static_assert((TSLOT * 4) % 128 == 0 && (OPSLOT * 4) % 128 == 0 && (SIDE * 4) % 128 == 0 &&
                      (USLOT * 4) % 128 == 0 && (NQ * CW * 4) % 128 == 0,
                  "tensor-copy destinations stay on 128 bytes");
    alignas(128) float v[RING][TSLOT];   // tile boxes: [q][row][DX]
    alignas(128) float pool[D][OPSLOT];  // operands [array][q][cell]; stage 2: k1 box at SIDE
    alignas(128) float upool[D][USLOT];  // profiles [n][cell]
    unsigned long long tbar[RING], obar[D];      // copies complete (bytes)
    F2 red[NT / 32][2 * MAXN];           // per-warp partial overlaps (integer digits)
    float redmax[NT / 32];
    const float *kp[7];                  // physical slope buffers in logical order
    const DenseMaps *maps;               // the launch's tensor maps (kernel parameter)
    int4 seg[MAX_BLOCK_SEGMENTS];        // this block's segments (x0, y0, z0, z1)
    int nseg;
};

// Tensor map `i` of the launch.
template <class SM>
__device__ __forceinline__ const void *tmap(const SM &sm, int i)
{
    return &sm.maps->map[i];
}

// Physical index of slope buffer p (select rather than index the kernel-parameter array).
__device__ __forceinline__ int slope_index(const Ctx &c, const float *p)
{
    int u = 0;
#pragma unroll
    for (int j = 1; j < 7; j++)
        if (p == c.k[j]) u = j;
    return u;
}

// Producer thread: the tile box of stream plane g (and at stage 2 the k1 box) into ring slot g mod
// RING.
template <int NS, int WY, bool HU, int S>
__device__ __forceinline__ void dense_issue_tile(const Ctx &c, DenseSmem<NS, WY, HU> &sm,
                                                 const float *mn, int g, Pipe &pp)
{
    using SM = DenseSmem<NS, WY, HU>;
    if (g >= pp.gend) return;
    cursor_seek(sm, pp.ci, g);
    const Cursor &cu = pp.ci;
    const int z = cu.z0 - 1 + (g - cu.off);
    const int r = g % SM::RING;
    const unsigned bytes = (unsigned)(SM::NQ * SM::P * 4) * (S == 2 ? 2u : 1u);
    mbar_arrive_expect_tx(&sm.tbar[r], bytes);
    const int src = S <= 2 ? TMT_M + (mn == c.m[0] ? 0 : 1) : TMT_MSV + (S & 1);
    tma_load4(sm.v[r], tmap(sm, src), cu.x0 - DOFF, cu.y0 - 1, z, &sm.tbar[r]);
    if (S == 2)
        tma_load4(sm.pool[g % SM::D] + SM::SIDE, tmap(sm, TMT_K + slope_index(c, sm.kp[0])),
                  cu.x0 - DOFF, cu.y0 - 1, z, &sm.tbar[r]);
}

// Producer thread: the operands (and profiles) of stream plane g into operand slot g mod D, or, for a
// halo plane, a plain arrival that completes the slot's phase.
template <int NS, int WY, bool HU, int S>
__device__ __forceinline__ void dense_issue_ops(const Ctx &c, DenseSmem<NS, WY, HU> &sm,
                                                const float *mn, int g, Pipe &pp)
{
    using SM = DenseSmem<NS, WY, HU>;
    constexpr int NO = n_ops(S);
    if (g >= pp.gend) return;
    cursor_seek(sm, pp.cr, g);
    const Cursor &cu = pp.cr;
    const int q = g - cu.off;
    const int s = g % SM::D;
    const bool inner = q >= 1 && q <= cu.np - 2;
    if (!inner || (NO == 0 && !HU)) {
        mbar_arrive(&sm.obar[s]);
        return;
    }
    const int z = cu.z0 - 1 + q;
    const unsigned bytes = (unsigned)(NO * SM::NQ * SM::CW * 4) +
                           (HU ? (unsigned)(c.nmodes * SM::CW * 4) : 0u);
    mbar_arrive_expect_tx(&sm.obar[s], bytes);
    const unsigned long long pol = l2_stream();
#pragma unroll
    for (int a = 0; a < NO; a++) {
        int mi;
        if (S == 7) mi = TMO_ES;
        else if (a == 0) mi = TMO_M + (mn == c.m[0] ? 0 : 1);
        else mi = TMO_K + slope_index(c, sm.kp[op_slope(S, a)]);
        tma_load4_hint(sm.pool[s] + a * SM::NQ * SM::CW, tmap(sm, mi), cu.x0, cu.y0, z,
                       &sm.obar[s], pol);
    }
    if (HU) tma_load4_hint(sm.upool[s], tmap(sm, TMO_U), cu.x0, cu.y0, z, &sm.obar[s], pol);
}

// Lane 0 of issuing warp k (of K): its share of the copies of one iteration, the tile box of
// stream plane gt (and at stage 2 its k1 box) and the operand boxes (and profiles) of stream
// plane go, dealt round-robin so that no warp carries all the issue work (every warp waits for
// the slowest at the plane's block barrier).  The issuer of the tile announces the tile bytes on
// its slot's barrier, the issuer of the first operand the operand bytes; a halo plane's operand
// phase is completed by a plain arrival.
template <int NS, int WY, bool HU, int S>
__device__ __forceinline__ void dense_issue_share(const Ctx &c, DenseSmem<NS, WY, HU> &sm,
                                                  const float *mn, int gt, int go, int k, int K,
                                                  Pipe &pp)
{
    using SM = DenseSmem<NS, WY, HU>;
    constexpr int NO = n_ops(S), NTC = S == 2 ? 2 : 1;
    const int nt = gt < pp.gend ? NTC : 0;
    int no = 0, zo = 0, xo = 0, yo = 0;
    bool inner = false;
    if (go < pp.gend) {
        cursor_seek(sm, pp.cr, go);
        const int q = go - pp.cr.off;
        inner = q >= 1 && q <= pp.cr.np - 2 && (NO > 0 || HU);
        no = inner ? NO + (HU ? 1 : 0) : 1;
        zo = pp.cr.z0 - 1 + q;
        xo = pp.cr.x0;
        yo = pp.cr.y0;
    }
    if (k >= nt + no) return;
    int zt = 0, xt = 0, yt = 0;
    if (nt) {
        cursor_seek(sm, pp.ci, gt);
        zt = pp.ci.z0 - 1 + (gt - pp.ci.off);
        xt = pp.ci.x0;
        yt = pp.ci.y0;
    }
    const int r = gt % SM::RING, s = go % SM::D;
    const unsigned long long pol = l2_stream();
    for (int i = k; i < nt + no; i += K) {
        if (i < nt) {
            if (i == 0) {
                mbar_arrive_expect_tx(&sm.tbar[r], (unsigned)(SM::NQ * SM::P * 4 * NTC));
                const int src = S <= 2 ? TMT_M + (mn == c.m[0] ? 0 : 1) : TMT_MSV + (S & 1);
                tma_load4(sm.v[r], tmap(sm, src), xt - DOFF, yt - 1, zt, &sm.tbar[r]);
            } else {
                tma_load4(sm.pool[gt % SM::D] + SM::SIDE,
                          tmap(sm, TMT_K + slope_index(c, sm.kp[0])), xt - DOFF, yt - 1, zt,
                          &sm.tbar[r]);
            }
            continue;
        }
        const int a = i - nt;
        if (!inner) {
            mbar_arrive(&sm.obar[s]);
            continue;
        }
        if (a == 0)
            mbar_arrive_expect_tx(&sm.obar[s], (unsigned)(NO * SM::NQ * SM::CW * 4) +
                                                   (HU ? (unsigned)(c.nmodes * SM::CW * 4) : 0u));
        if (a < NO) {
            int mi;
            if (S == 7) mi = TMO_ES;
            else if (a == 0) mi = TMO_M + (mn == c.m[0] ? 0 : 1);
            else mi = TMO_K + slope_index(c, sm.kp[op_slope(S, a)]);
            tma_load4_hint(sm.pool[s] + a * SM::NQ * SM::CW, tmap(sm, mi), xo, yo, zo,
                           &sm.obar[s], pol);
        } else {
            tma_load4_hint(sm.upool[s], tmap(sm, TMO_U), xo, yo, zo, &sm.obar[s], pol);
        }
    }
}

// Stage 2: the values m_2 = m_n + h a_21 k_1 of every position of plane g's tile box (its copies
// are complete), spread over the block's threads; the block barrier that follows publishes them.
template <int NS, int WY, bool HU, int S>
__device__ __forceinline__ void dense_tile_combine(DenseSmem<NS, WY, HU> &sm, const Coef &cf, int g,
                                                   const Pipe &pp)
{
    using SM = DenseSmem<NS, WY, HU>;
    if (S != 2 || g >= pp.gend) return;
    float *v = sm.v[g % SM::RING];
    const float *side = sm.pool[g % SM::D] + SM::SIDE;
    const float c21 = cf.cf[1][0];
    for (int e = threadIdx.x; e < SM::NQ * SM::P; e += SM::NT) v[e] = fmaf(c21, side[e], v[e]);
}

// RHS of this thread's cell of stream plane p (ring slots p-1, p, p+1) at box plane z, then the
// combine of the next stage value (stages 2..6), the error partial (stage 6) or the error
// estimate and the renormalised new state (stage 7); the stores and their order are those of
// compute_cell in cmx_stage.cuh.
template <int NS, int WY, bool HU, int S>
__device__ __forceinline__ void dense_cell(const Ctx &c, DenseSmem<NS, WY, HU> &sm, float *kout,
                                           float *mnew, const Coef &cf, int p, int x0, int y0,
                                           int z, int tslot, int rslot, Acc &acc)
{
    // the plane's operands (and profiles) are waited for where they are first used: the copies
    // then have the stencil's time to land as well
    using SMT = DenseSmem<NS, WY, HU>;
    auto wait_ops = [&]() {
        mbar_wait(c, &sm.obar[p % SMT::D], (unsigned)((p / SMT::D) & 1), 23);
    };
    using SM = DenseSmem<NS, WY, HU>;
    constexpr int NQ = SM::NQ, R = SM::RING, CW = SM::CW, P = SM::P, NO = n_ops(S);
    const int i = threadIdx.x, lane = i & 31, row = i >> 5;
    const int x = x0 + lane, y = y0 + row;
    if (x >= c.nx || y >= c.ny) return;
    const int idx = (z * c.ny + y) * c.nxs + x;
    if (!idx_ok(c, idx, c.ncell, 20)) return;
    if (S >= 2 && rslot >= 0 && !idx_ok(c, rslot, c.rec_steps, 7)) return;
    if ((S == 1 || S == 7) && tslot >= 0 && !idx_ok(c, tslot, c.traj_slots, 8)) return;
    const float *vp = sm.v[(p + R - 1) % R], *vc = sm.v[p % R], *vn = sm.v[(p + 1) % R];
    const float *op = sm.pool[p % SM::D];
    const int e = (1 + row) * DX + DOFF + lane;
    // neighbours inside the box (the copies fill positions outside it with 0)
    const float nxc = (x > 0 ? 1.f : 0.f) + (x + 1 < c.nx ? 1.f : 0.f);
    const float nyc = (y > 0 ? 1.f : 0.f) + (y + 1 < c.ny ? 1.f : 0.f);
    const float nzc = (z > 0 ? 1.f : 0.f) + (z + 1 < c.nz ? 1.f : 0.f);

    float m[NS][3], B[NS][3];
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = s * 3 + k;
            const float *a = vc + q * P;
            const float cen = a[e];
            m[s][k] = cen;
            // exchange: sum over present neighbours of (m_j - m_i) / c_d^2 (absent ones hold 0)
            B[s][k] = c.wx * (a[e - 1] + a[e + 1] - nxc * cen) +
                      c.wy * (a[e - DX] + a[e + DX] - nyc * cen) +
                      c.wz * (vp[q * P + e] + vn[q * P + e] - nzc * cen);
        }
    if (HU) wait_ops();
    float ucell[MAXN];
#pragma unroll
    for (int n = 0; n < MAXN; n++)
        ucell[n] = (HU && n < c.nmodes) ? sm.upool[p % SM::D][n * CW + i] : 1.f;
    const float bdem[3] = {0.f, 0.f, 0.f};
    float kv[NS][3];
    cell_slope<NS, HU>(c, cf, m, B, ucell, bdem, acc, kv);

#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = s * 3 + k;
            kout[(size_t)q * c.ncell + idx] = kv[s][k];
            if (S >= 2 && rslot >= 0)
                c.rec_m[((size_t)rslot * 6 + (S >= 2 ? S - 2 : 0)) * NQ * c.ncell +
                        (size_t)q * c.ncell + idx] = m[s][k];
        }
    if ((S == 1 || S == 7) && tslot >= 0) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            const float *mm = m[s];
            const float r = S == 7 ? rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]) : 1.f;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const size_t o = (size_t)tslot * NQ * c.ncell + (size_t)(s * 3 + k) * c.ncell + idx;
                c.traj_m[o] = mm[k] * r;
                c.traj_k[o] = kv[s][k];
            }
        }
    }
    if (!HU && (S >= 2 && S <= 7)) wait_ops();
    if (S >= 2 && S <= 6 && !c.stage_only) {
        // next stage value m_{S+1} = m_n + sum_j (h a_{S+1,j}) k_j, k_S last; error partial
        const unsigned long long keep = l2_keep();
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int q = s * 3 + k;
                float a = op[(0 * NQ + q) * CW + i], es = 0.f;
#pragma unroll
                for (int o = 1; o < NO; o++) {
                    const int j = op_slope(S, o);
                    const float kj = op[(o * NQ + q) * CW + i];
                    a = fmaf(cf.cf[S][j], kj, a);
                    if (S == 6) es = fmaf(cf.e[j], kj, es);
                }
                a = fmaf(cf.cf[S][S - 1], kv[s][k], a);
                es = fmaf(cf.e[5], kv[s][k], es);
                st_hint(c.msv[(S + 1) & 1] + (size_t)q * c.ncell + idx, a, keep);
                if (S == 6) st_hint(c.es + (size_t)q * c.ncell + idx, es, keep);
            }
    }
    if (S == 7) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            const float *mm = m[s];
            const float r = rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int q = s * 3 + k;
                const float e7 = cf.h * fmaf(cf.e[6], kv[s][k], op[q * CW + i]);
                acc.emax = nanmax(acc.emax, fabsf(e7));
                mnew[(size_t)q * c.ncell + idx] = mm[k] * r;
            }
        }
    }
}

// Start stage S's stream: (re)initialise the slot barriers, then the producer issues the first
// planes' copies (tiles of planes 0, 1 and, except at stage 2, 2; operands of planes 0, 1).  At
// stage 2 plane 2's tile waits for the combine of plane 0, whose k1 box shares its buffer.
template <int NS, int WY, bool HU, int S>
__device__ void dense_begin(const Ctx &c, DenseSmem<NS, WY, HU> &sm, const float *mn, Pipe &pp)
{
    using SM = DenseSmem<NS, WY, HU>;
    pp.gend = 0;
    for (int t = 0; t < sm.nseg; t++) pp.gend += sm.seg[t].w - sm.seg[t].z + 2;
    pp.nq = 0;
    if (sm.nseg == 0) return;
    pp.ci = cursor_start(sm);
    pp.cr = pp.ci;
    pp.cc = pp.ci;
    __syncthreads();   // the previous stage may still read the shared buffers
    if (threadIdx.x == SM::PROD) {
        for (int r = 0; r < SM::RING; r++) mbar_init(&sm.tbar[r], 1);
        for (int s = 0; s < SM::D; s++) mbar_init(&sm.obar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == SM::PROD) {
        fence_proxy_async_global();
        dense_issue_tile<NS, WY, HU, S>(c, sm, mn, 0, pp);
        dense_issue_tile<NS, WY, HU, S>(c, sm, mn, 1, pp);
        if (S != 2) dense_issue_tile<NS, WY, HU, S>(c, sm, mn, 2, pp);
        dense_issue_ops<NS, WY, HU, S>(c, sm, mn, 0, pp);
        dense_issue_ops<NS, WY, HU, S>(c, sm, mn, 1, pp);
    }
    __syncwarp();
}

// Run stage S's stream to its end (see the file comment for the schedule).  Every issued copy is
// waited for before the stream ends: tiles of all planes, operands of the interior planes (the
// halo planes' operand phases carry no copies).
template <int NS, int WY, bool HU, int S>
__device__ void dense_run(const Ctx &c, DenseSmem<NS, WY, HU> &sm, float *kout, const float *mn,
                          float *mnew, const Coef &cf, Pipe &pp, int tslot, int rslot, Acc &acc)
{
    using SM = DenseSmem<NS, WY, HU>;
    constexpr int R = SM::RING, D = SM::D;
    const int gend = pp.gend;
    if (sm.nseg == 0) return;
    mbar_wait(c, &sm.tbar[0], 0, 21);
    mbar_wait(c, &sm.tbar[1], 0, 21);
    if (S == 2) {
        dense_tile_combine<NS, WY, HU, S>(sm, cf, 0, pp);
        dense_tile_combine<NS, WY, HU, S>(sm, cf, 1, pp);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == SM::PROD) dense_issue_tile<NS, WY, HU, S>(c, sm, mn, 2, pp);
        __syncwarp();
    }
    for (int p = 1; p <= gend - 2; p++) {
        mbar_wait(c, &sm.tbar[(p + 1) % R], (unsigned)(((p + 1) / R) & 1), 22);
        dense_tile_combine<NS, WY, HU, S>(sm, cf, p + 1, pp);
        // stage 2 wrote the tile in place: order those writes before later copies into the slot
        // (reads alone are ordered by the block barrier)
        if (S == 2) fence_proxy_async_smem();
        __syncthreads();
        {
            // issuing warps 1 .. NW-1 (warp 0 runs the controller between stages)
            const int w = threadIdx.x >> 5;
            if ((threadIdx.x & 31) == 0 && w >= 1)
                dense_issue_share<NS, WY, HU, S>(c, sm, mn, p + 2, p + 1, w - 1, SM::NT / 32 - 1,
                                                 pp);
        }
        __syncwarp();
        cursor_seek(sm, pp.cc, p);
        const int q = p - pp.cc.off;
        if (q >= 1 && q <= pp.cc.np - 2) {
            dense_cell<NS, WY, HU, S>(c, sm, kout, mnew, cf, p, pp.cc.x0, pp.cc.y0,
                                      pp.cc.z0 - 1 + q, tslot, rslot, acc);
        }
    }
    // this stage's stores are read by the next stages' tensor copies (after the grid barrier)
    fence_proxy_async_global();
}

// Engine-facing names of the dense stage code (overloads by shared-memory type).
template <int S, int NS, int WY, bool HU>
__device__ __forceinline__ void stage_begin(const Ctx &c, DenseSmem<NS, WY, HU> &sm,
                                            const float *mn, Pipe &pp)
{
    dense_begin<NS, WY, HU, S>(c, sm, mn, pp);
}

template <int S, int NS, int WY, bool HU>
__device__ __forceinline__ void stage_run(const Ctx &c, DenseSmem<NS, WY, HU> &sm, float *kout,
                                          const float *mn, float *mnew, const Coef &cf, Pipe &pp,
                                          int tslot, int rslot, Acc &acc)
{
    dense_run<NS, WY, HU, S>(c, sm, kout, mn, mnew, cf, pp, tslot, rslot, acc);
}

template <int NS, int WY, bool HU>
__device__ void stage_cache_rows(const Ctx &, DenseSmem<NS, WY, HU> &)
{
}

template <int NS, int WY, bool HU>
__host__ __device__ constexpr int cells_per_thread(const DenseSmem<NS, WY, HU> *)
{
    return 1;
}

}  // namespace cmx
