// Device code of one Dormand-Prince stage over the tiles of a masked grid (sm_103a).
//
// Stage S computes, for every magnetic cell, the field at the stage value m_S,
//   B    = exchange(m_S) + anisotropy + Zeeman + demag + inter-sublattice + B_rf(a_S)
//   k_S  = -gamma/(1+alpha^2) [ m_S x B + alpha m_S x (m_S x B) ]      (LLG, Sec. II A)
// and the block partial sums of the overlaps u_n (m_x - i m_y) (Eq. (18)); then, with k_S still
// in registers, it combines the cell's NEXT stage value and stores it:
//   m_{S+1} = m_n + h sum_{j<=S} a_{S+1,j} k_j                      (S = 2..6; S = 6 gives the
//                                                                     5th-order point Y_7)
// Stage S+1 reads these stored values for its tile and its one-cell halo, so a halo cell's
// stage value is read (12 bytes per sublattice, mostly from L2: the neighbouring tiles wrote it
// during the previous stage) instead of being recombined from m_n and all earlier slopes of that
// cell.  The step size of an attempt is fixed only by the previous attempt's decision, so stage 2
// forms m_2 = m_n + h a_21 k_1 itself for every tile position; stage 1 reads m_n.  Stage 6 also
// stores the error partial sum_{j<=6} E_j k_j, and stage 7 adds E_7 k_7 to it:
// e_m = h sum_j E_j k_j, and writes the renormalised 5th-order point.
//
// A tile is WX x WY cells (one warp per x-row, every thread computes a cell) with a one-cell rim
// that the first threads of the block load as well; blocks march through their columns plane by
// plane.  Stage values of the tile and rim and the thread's own operands of the next combine
// arrive by asynchronous copies (cp.async) several planes ahead; one __syncthreads per plane
// publishes a plane's tile, and the 6-neighbour stencil reads only shared memory.  Cells are
// stored compactly per (y, z) row between the first and the last magnetic x of the row; the row
// table gives the offset.
#pragma once

#include "cmx_internal.cuh"

namespace cmx {

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    return *(const volatile int *)p;
}

// Index check of the bounds-checked build (CMX_CHECK): true if 0 <= i < n; otherwise the run
// stops with CMX_ECHECK, the site and the index are recorded, and the caller skips the access.
// Always true in the plain build.
__device__ __forceinline__ bool idx_ok(const Ctx &c, long long i, long long n, int site)
{
#if CMX_CHECK
    if (i >= 0 && i < n) return true;
    if (atomicCAS(&c.ctl->status, 0, (int)CMX_ECHECK) == 0) {
        c.ctl->timeout_where = site;
        c.ctl->check_value = i;
    }
    return false;
#else
    (void)c;
    (void)i;
    (void)n;
    (void)site;
    return true;
#endif
}

// max that propagates NaN (a NaN error estimate must reach the controller)
__device__ __forceinline__ float nanmax(float a, float b)
{
    return (a != a || b != b) ? __int_as_float(0x7fffffff) : fmaxf(a, b);
}

// The mode constants of mode n (MC doubles) from the context (select rather than index the
// kernel-parameter arrays, which keeps them out of local memory).
__device__ __forceinline__ void mode_constants(const Ctx &c, int n, double *out)
{
    double v[MC] = {c.omega[0], c.kappa[0], c.gre[0], c.gim[0], c.gbre[0], c.gbim[0], c.kerr[0]};
#pragma unroll
    for (int u = 1; u < MAXN; u++)
        if (n == u) {
            v[0] = c.omega[u];
            v[1] = c.kappa[u];
            v[2] = c.gre[u];
            v[3] = c.gim[u];
            v[4] = c.gbre[u];
            v[5] = c.gbim[u];
            v[6] = c.kerr[u];
        }
#pragma unroll
    for (int q = 0; q < MC; q++) out[q] = v[q];
}

// Operand arrays of the combine that ends stage S (1-based), read for the thread's own cell:
// stages 2..6 read m_n (array 0) and the earlier slopes k_j, j < S, with a nonzero coupling
// a_{S+1,j} (k_S itself is in registers); stage 7 reads the error partial stored by stage 6.
__host__ __device__ constexpr int n_ops(int S)
{
    if (S <= 1) return 0;
    if (S == 7) return 1;
    int n = 1;
    for (int j = 0; j < S - 1; j++) n += dp_a(S, j) != 0.0 ? 1 : 0;
    return n;
}

// Slope (0-based) held by operand array a >= 1 of stage S.
__host__ __device__ constexpr int op_slope(int S, int a)
{
    int n = 0;
    for (int j = 0; j < S - 1; j++)
        if (dp_a(S, j) != 0.0) {
            n++;
            if (n == a) return j;
        }
    return -1;
}

// The error partial of stage 6 uses the same slopes as the 5th-order point (E_2 = a_72 = 0).
__host__ __device__ constexpr bool error_slopes_match()
{
    for (int j = 0; j < 6; j++)
        if ((dp_e(j) != 0.0) != (dp_a(6, j) != 0.0)) return false;
    return true;
}
static_assert(error_slopes_match(), "stage 6 forms Y_7 and the error partial from one operand set");

// Arrays per tile position: stage 2 loads m_n and k_1 and combines them; the other stages load
// one stage value (m_n at stage 1, the stored m_S otherwise).
__host__ __device__ constexpr int n_tile(int S)
{
    return S == 2 ? 2 : 1;
}

// Compensated FP32 pair ("double-float"): value = hi + lo, about 44 significant bits.  Used for
// the fixed-order sums of the adjoint's reverse sweep.
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);   // exact rounding error of a.hi + b.hi
    e += a.lo + b.lo;
    const float hi = s + e;
    return {hi, e - (hi - s)};
}

__device__ __forceinline__ F2 f2_shfl_xor(F2 a, int o)
{
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Asynchronous 4-byte global -> shared copy (LDGSTS), its group commit and wait.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}

// L2 eviction-priority policies: stored stage values are kept in L2 from the stage that writes
// them to the next one that reads them (evict_last); the operands streamed once per stage from
// DRAM are the first to leave (evict_first).
__device__ __forceinline__ unsigned long long l2_keep()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ unsigned long long l2_stream()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void cp_async4_hint(void *smem, const void *gmem, unsigned long long pol)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem),
                 "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void st_hint(float *gmem, float v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(gmem), "f"(v), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Row-table entries cached for the first planes of a block's stream.
constexpr int ROWC = 16;

// Shared memory of a block of 32 x WY threads whose tile is CX x WY cells: every thread owns a
// "unit" of CPT = CX / 32 consecutive x-cells of one tile row (CPT = 1 or 2).  The tile of a
// plane holds PXS x PY positions: the tile's cells at columns OFF .. OFF+CX-1 of rows 1 .. WY,
// the one-cell rim at rows 0 and PY-1 and at columns OFF-1 and OFF+CX (OFF = CPT keeps every unit
// aligned to its size).  RING planes of stage values and presence (p-1, p, p+1 read by the
// stencil of plane p, later planes in flight).  The operand pool holds, per plane in flight, the
// thread's own operands of the next combine ([array][q][cell]) and, at stage 2, the slope k_1 of
// the tile positions ([q][position]); with mode profiles their values of the thread's unit.
template <int NS, int CX, int WY, bool HU>
struct StageSmem {
    static constexpr int CPT = CX / 32;                   // cells per thread
    static constexpr int NT = 32 * WY;                    // threads
    static constexpr int CW = CX * WY;                    // cells of a tile plane
    static constexpr int OFF = CPT;
    static constexpr int PXS = CX + 2 * OFF, PY = WY + 2, P = PXS * PY;
    static constexpr int NRU = 64;                        // rim units: rows 0 and PY-1
    static constexpr int NRS = 2 * PY;                    // rim singles: columns OFF-1, OFF+CX
    static constexpr int NQ = NS * 3;
    static constexpr int NAMAX = 5;                       // m_n + at most four slopes
    static constexpr int D = 2;                           // planes in flight
    static constexpr int RING = D + 2;                    // tile slots
    static constexpr int OIX = D + 1;                     // own-index slots
    static constexpr int OPSLOT = NAMAX * NQ * CW;        // operand slot (D of them)
    static constexpr int USLOT = HU ? MAXN * CW : 0;      // profile slot (D of them)
    static_assert(CX == 32, "one cell per thread (64-wide two-cell tiles measured slower)");
    static_assert(2 * NQ * CW + NQ * P <= OPSLOT, "stage-2 slot");
    static_assert(NRU + NRS <= NT, "rim loads need one thread each");
    static_assert(P % 2 == 0 && CW % 2 == 0 && OPSLOT % 4 == 0, "units stay 8-byte aligned");
    alignas(16) float pool[D * OPSLOT];
    alignas(16) float upool[D * USLOT + 4];
    alignas(16) float v[RING][NQ + 1][P];   // stage values of the tile positions, presence in row NQ
    int oidx[OIX][NT];            // compact index of the thread's first cell of a plane in flight
                                  // (-1: no magnetic cell, or a halo plane)
    F2 red[NT / 32][2 * MAXN];    // per-warp partial overlaps (integer digits)
    float redmax[NT / 32];
    const float *kp[7];           // physical slope buffers in logical order
    int2 rows[8][PY];             // row-table entries of the tile rows, by plane mod 8
    int2 rowc[ROWC][PY];          // the same for the first ROWC planes of the stream (every
                                  // stage starts there), filled once per launch
    int4 seg[MAX_BLOCK_SEGMENTS]; // this block's segments (x0, y0, z0, z1)
    int nseg;
};

// Position of a cursor in a block's stream of planes: segment t, whose first plane is stream
// position `off`; the segment has np = z1 - z0 + 2 planes (z0-1 .. z1).
struct Cursor {
    int t, off, np, x0, y0, z0;
};

template <class SM>
__device__ __forceinline__ void cursor_seek(const SM &sm, Cursor &cu, int g)
{
    while (g >= cu.off + cu.np && cu.t + 1 < sm.nseg) {
        cu.off += cu.np;
        cu.t++;
        const int4 T = sm.seg[cu.t];
        cu.x0 = T.x;
        cu.y0 = T.y;
        cu.z0 = T.z;
        cu.np = T.w - T.z + 2;
    }
}

template <class SM>
__device__ __forceinline__ Cursor cursor_start(const SM &sm)
{
    const int4 T = sm.seg[0];
    return Cursor{0, 0, T.w - T.z + 2, T.x, T.y, T.z};
}

// Per-thread accumulators of one stage.
struct Acc {
    float re[MAXN], im[MAXN];
    float emax;
};

// FP32 stage coefficients of the current attempt: cf[S-1][j] = h a_Sj for every stage S, e[j] =
// E_j, h, and the feedback field per unit profile of each mode at the current stage,
// hrf[n] = (2/gamma) Re[g~_n a_{n,S}] (Eq. (5), (13)).
struct Coef {
    float cf[7][6];
    float e[7];
    float h;
    float hrf[MAXN];
};

// Compact index of box cell x in a row given its row-table entry, or -1.  The entry holds the
// storage offset of the row's first stored cell, which is x = xs rounded down to ROW_ALIGN, and
// the magnetic span [xs, xe); cells inside the span that are not magnetic (holes) are marked in
// the active bitmask (NULL: no holes).
__device__ __forceinline__ int row_index(const Ctx &c, int2 r, int x)
{
    const int xs = r.y & 0xffff, xe = (int)((unsigned)r.y >> 16);
    if (x < xs || x >= xe) return -1;
    const int idx = r.x + (x - (xs & ~(ROW_ALIGN - 1)));
    if (c.active && !((__ldg(&c.active[idx >> 5]) >> (idx & 31)) & 1u)) return -1;
    return idx;
}

__device__ __forceinline__ int2 row_entry(const Ctx &c, int y, int z)
{
    if ((unsigned)y >= (unsigned)c.ny || (unsigned)z >= (unsigned)c.nz) return make_int2(0, 0);
    return __ldg(&c.rows[z * c.ny + y]);
}

// Storage index of the unit of CPT cells that starts at box x (a multiple of CPT) in a row, or
// -1 if the unit lies outside the row's stored span (whose ends are multiples of ROW_ALIGN, so
// a unit is either inside or outside); pres[k] = 1 if cell x + k is magnetic.
template <int CPT>
__device__ __forceinline__ int unit_index(const Ctx &c, int2 r, int x, float (&pres)[CPT])
{
    const int xs = r.y & 0xffff, xe = (int)((unsigned)r.y >> 16);
    const int xa = xs & ~(ROW_ALIGN - 1), xb = (xe + ROW_ALIGN - 1) & ~(ROW_ALIGN - 1);
#pragma unroll
    for (int k = 0; k < CPT; k++) pres[k] = 0.f;
    if (x < xa || x >= xb) return -1;
    const int idx = r.x + (x - xa);
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        bool on = x + k >= xs && x + k < xe;
        if (on && c.active) on = (__ldg(&c.active[(idx + k) >> 5]) >> ((idx + k) & 31)) & 1u;
        pres[k] = on ? 1.f : 0.f;
    }
    return idx;
}

// Asynchronous global -> shared copy of one unit (4 bytes per cell).
template <int CPT>
__device__ __forceinline__ void cp_async_unit(void *smem, const void *gmem)
{
    static_assert(CPT == 1, "one cell per unit");
    cp_async4(smem, gmem);
}

// The CPT values of a unit in shared memory.
template <int CPT>
__device__ __forceinline__ void unit_load(const float *p, float (&o)[CPT])
{
#pragma unroll
    for (int u = 0; u < CPT; u++) o[u] = p[u];
}

// Copy-pipeline state of one stage: cursors for row loading (cr) and copy issue (ci), the next
// plane to issue, the stream length, and the thread's tile positions: its own unit (eo) and the
// rim element it loads (er, -1: none), a unit (rk = 1) or a single cell (rk = 2) at row rr and
// column offset rc from the tile's x0 (rc in box cells).
struct Pipe {
    Cursor cr, ci, cc;
    int nq, gend;
    int eo, er, rr, rc, rk;
};

// Source of the tile values of stage S: m_n (S = 1, 2) or the stored stage value.
template <int S>
__device__ __forceinline__ const float *tile_source(const Ctx &c, const float *mn)
{
    return S <= 2 ? mn : c.msv[S & 1];
}

// Source of operand array a of stage S.
template <class SM, int S>
__device__ __forceinline__ const float *op_source(const Ctx &c, const SM &sm, const float *mn,
                                                  int a)
{
    if (S == 7) return c.es;
    if (a == 0) return mn;
    return sm.kp[op_slope(S, a)];
}

// Copies of U tile positions e .. e+U-1 (stored from compact index idx, or -1: outside the
// row's stored span) of stream plane g into ring slot rs: stage values (and at stage 2 the slope
// k_1 into the side array), presence written directly.  Inactive cells inside a stored span hold
// 0 in every array, so a copied unit needs no masking; a position outside is zero-filled.
template <class SM, int S, int U>
__device__ __forceinline__ void load_positions(const Ctx &c, SM &sm, const float *tsrc, int rs,
                                               float *side, int e, int idx, const float (&pres)[U])
{
    constexpr int NQ = SM::NQ, P = SM::P;
    if (!idx_ok(c, e, P - U + 1, 1) || !idx_ok(c, rs, SM::RING, 2)) return;
    if (idx >= 0 && !idx_ok(c, idx, (long long)c.ncell - U + 1, 3)) idx = -1;
    if (idx >= 0) {
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            cp_async_unit<U>(&sm.v[rs][k][e], tsrc + (size_t)k * c.ncell + idx);
            if (S == 2) cp_async_unit<U>(side + k * P + e, sm.kp[0] + (size_t)k * c.ncell + idx);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NQ; k++)
#pragma unroll
            for (int u = 0; u < U; u++) {
                sm.v[rs][k][e + u] = 0.f;
                if (S == 2) side[k * P + e + u] = 0.f;
            }
    }
#pragma unroll
    for (int u = 0; u < U; u++) sm.v[rs][NQ][e + u] = pres[u];
}

// Copies of stream plane g, in two commit groups: first the tile (the thread's unit and, for the
// first NRU + NRS threads, one rim unit or single) with the presence flags and the own compact
// index, later the thread's own operands of the stage's combine (and profiles) on planes
// interior to their segment.  Both commit one group (possibly empty).
template <int NS, int CX, int WY, bool HU, int S>
__device__ __forceinline__ void issue_tile(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm,
                                           const float *mn, int g, Pipe &pp)
{
    using SM = StageSmem<NS, CX, WY, HU>;
    constexpr int NQ = SM::NQ, CPT = SM::CPT;
    const int i = threadIdx.x;
    if (g < pp.gend) {
        cursor_seek(sm, pp.ci, g);
        const Cursor &cu = pp.ci;
        const int q = g - cu.off;
        const bool inner = q >= 1 && q <= cu.np - 2;
        const int rs = g % SM::RING;
        float *side = sm.pool + (size_t)(g % SM::D) * SM::OPSLOT + n_ops(2) * NQ * SM::CW;
        const float *tsrc = tile_source<S>(c, mn);
        const int2 *rw = sm.rows[g & 7];
        float pres[CPT];
        const int idx = unit_index<CPT>(c, rw[i / 32 + 1], cu.x0 + CPT * (i % 32), pres);
        load_positions<SM, S, CPT>(c, sm, tsrc, rs, side, pp.eo, idx, pres);
        bool any = false;
#pragma unroll
        for (int u = 0; u < CPT; u++) any |= pres[u] != 0.f;
        sm.oidx[g % SM::OIX][i] = (inner && any) ? idx : -1;
        if (pp.rk == 1) {
            float rp[CPT];
            const int ridx = unit_index<CPT>(c, rw[pp.rr], cu.x0 + pp.rc, rp);
            load_positions<SM, S, CPT>(c, sm, tsrc, rs, side, pp.er, ridx, rp);
        } else if (pp.rk == 2) {
            float rp[1];
            const int ridx = row_index(c, rw[pp.rr], cu.x0 + pp.rc);
            rp[0] = ridx >= 0 ? 1.f : 0.f;
            load_positions<SM, S, 1>(c, sm, tsrc, rs, side, pp.er, ridx, rp);
        }
    }
    cp_async_commit();
}

template <int NS, int CX, int WY, bool HU, int S>
__device__ __forceinline__ void issue_ops(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm,
                                          const float *mn, int g, const Pipe &pp)
{
    using SM = StageSmem<NS, CX, WY, HU>;
    constexpr int NQ = SM::NQ, CW = SM::CW, CPT = SM::CPT, NO = n_ops(S);
    const int i = threadIdx.x;
    if (g < pp.gend) {
        const int oi = sm.oidx[g % SM::OIX][i];
        if (oi >= 0 && idx_ok(c, oi, (long long)c.ncell - CPT + 1, 4)) {
            float *slot = sm.pool + (size_t)(g % SM::D) * SM::OPSLOT;
            const unsigned long long pol = l2_stream();
#pragma unroll
            for (int a = 0; a < NO; a++) {
                const float *src = op_source<SM, S>(c, sm, mn, a);
#pragma unroll
                for (int k = 0; k < NQ; k++)
                    cp_async4_hint(slot + (a * NQ + k) * CW + CPT * i,
                                   src + (size_t)k * c.ncell + oi, pol);
            }
            if (HU) {
                float *us = sm.upool + (size_t)(g % SM::D) * SM::USLOT;
#pragma unroll
                for (int n = 0; n < MAXN; n++)
                    if (n < c.nmodes)
                        cp_async_unit<CPT>(us + n * CW + CPT * i, c.u + (size_t)n * c.ncell + oi);
            }
        }
    }
    cp_async_commit();
}

// Stage 2: the tile values m_2 = m_n + h a_21 k_1 of the thread's positions of plane g (the
// copies of plane g are complete; only this thread wrote these positions).
template <int NS, int CX, int WY, bool HU, int S>
__device__ __forceinline__ void tile_combine(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm,
                                             const Coef &cf, int g, const Pipe &pp)
{
    using SM = StageSmem<NS, CX, WY, HU>;
    constexpr int NQ = SM::NQ, P = SM::P, CPT = SM::CPT;
    if (S != 2 || g >= pp.gend) return;
    const int rs = g % SM::RING;
    const float *side = sm.pool + (size_t)(g % SM::D) * SM::OPSLOT + n_ops(2) * NQ * SM::CW;
    const float c21 = cf.cf[1][0];
    const int nr = pp.rk == 1 ? CPT : (pp.rk == 2 ? 1 : 0);
    if (!idx_ok(c, pp.eo, P - CPT + 1, 9) || (nr && !idx_ok(c, pp.er, P - nr + 1, 10))) return;
#pragma unroll
    for (int k = 0; k < NQ; k++) {
#pragma unroll
        for (int u = 0; u < CPT; u++) {
            const int e = pp.eo + u;
            sm.v[rs][k][e] = fmaf(c21, side[k * P + e], sm.v[rs][k][e]);
        }
        for (int u = 0; u < nr; u++) {
            const int e = pp.er + u;
            sm.v[rs][k][e] = fmaf(c21, side[k * P + e], sm.v[rs][k][e]);
        }
    }
}

// Slope of one cell from its stage value m and exchange field B (both sublattices): adds the
// local fields (uniaxial anisotropy, Zeeman, diagonal demag of the total moment or the full
// demag field bdem of the cell (zero unless Ctx::fd; dmg is zero then),
// inter-sublattice -B_E m_other) and the cavity feedback field x sum_n u_n (2/gamma)
// Re[g~_n a_n] (Eq. (5), (13)) to B, accumulates the overlap partial sums of the net moment
// (m1 + m2)/2 with the same profile values (Eq. (18)), and returns the Landau-Lifshitz slope
// k = -gamma/(1+alpha^2) [m x B + alpha m x (m x B)].
template <int NS, bool HU>
__device__ __forceinline__ void cell_slope(const Ctx &c, const Coef &cf, const float (&m)[NS][3],
                                           float (&B)[NS][3], const float *ucell,
                                           const float (&bdem)[3], Acc &acc, float (&kv)[NS][3])
{
    float mt[3];
#pragma unroll
    for (int k = 0; k < 3; k++) mt[k] = (NS == 2) ? (m[0][k] + m[1][k]) : m[0][k];
    const float hx = (NS == 2) ? 0.5f * mt[0] : mt[0];
    const float hy = (NS == 2) ? 0.5f * mt[1] : mt[1];
    float brf = 0.f;
#pragma unroll
    for (int n = 0; n < MAXN; n++) {
        if (n >= c.nmodes) break;   // leaves the unrolled chain after the problem's modes
        const float un = HU ? ucell[n] : 1.f;
        brf = fmaf(un, cf.hrf[n], brf);
        acc.re[n] = fmaf(un, hx, acc.re[n]);
        acc.im[n] = fmaf(-un, hy, acc.im[n]);
    }
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const float mk = m[s][0] * c.ku[0] + m[s][1] * c.ku[1] + m[s][2] * c.ku[2];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float b = B[s][k] + c.anis * mk * c.ku[k] + c.B0[k] - c.dmg[k] * mt[k] + bdem[k];
            if (NS == 2) b -= c.BE * m[1 - s][k];
            B[s][k] = b;
        }
        B[s][0] += brf;
    }
    // LLG torque, Landau-Lifshitz form
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const float *mm = m[s], *b = B[s];
        const float t1x = mm[1] * b[2] - mm[2] * b[1];
        const float t1y = mm[2] * b[0] - mm[0] * b[2];
        const float t1z = mm[0] * b[1] - mm[1] * b[0];
        const float t2x = mm[1] * t1z - mm[2] * t1y;
        const float t2y = mm[2] * t1x - mm[0] * t1z;
        const float t2z = mm[0] * t1y - mm[1] * t1x;
        kv[s][0] = c.pre * fmaf(c.alpha, t2x, t1x);
        kv[s][1] = c.pre * fmaf(c.alpha, t2y, t1y);
        kv[s][2] = c.pre * fmaf(c.alpha, t2z, t1z);
    }
}

// RHS of this thread's unit of plane p (ring slots: p-1, p, p+1), then the combine of the next
// stage value from k_S and the operands in flight (stages 2..6), the error partial (stage 6), or
// the error estimate and the renormalised new state (stage 7).  Accumulates the overlap sums and
// the error maximum over the unit's magnetic cells; a non-magnetic cell of the unit gets 0 in
// every output (inactive cells hold 0 in every array).
template <int NS, int CX, int WY, bool HU, int S>
__device__ __forceinline__ void compute_cell(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm,
                                             float *kout, float *mnew, const Coef &cf, int p,
                                             int tslot, int rslot, const Pipe &pp, Acc &acc)
{
    using SM = StageSmem<NS, CX, WY, HU>;
    constexpr int NQ = SM::NQ, R = SM::RING, PXS = SM::PXS, CW = SM::CW, CPT = SM::CPT;
    constexpr int NO = n_ops(S), P = SM::P;
    const int i = threadIdx.x;
    const int idx = sm.oidx[p % SM::OIX][i];
    if (idx < 0) return;
    const int sp = (p + R - 1) % R, sc = p % R, sn = (p + 1) % R;
    const int e = pp.eo;
    if (!idx_ok(c, idx, (long long)c.ncell - CPT + 1, 5) || !idx_ok(c, e - PXS, P - 2 * PXS - CPT + 1, 6))
        return;
    if (S >= 2 && rslot >= 0 && !idx_ok(c, rslot, c.rec_steps, 7)) return;
    if ((S == 1 || S == 7) && tslot >= 0 && !idx_ok(c, tslot, c.traj_slots, 8)) return;
    const float *op = sm.pool + (size_t)(p % SM::D) * SM::OPSLOT;
    const int oc = CPT * i;   // the unit's first cell in the operand slot
    const float *pr = sm.v[sc][NQ];

    // presence of the unit's cells and their neighbour counts per axis
    float here[CPT], nx_[CPT], ny_[CPT], nz_[CPT];
    {
        float a[CPT], b[CPT], z0[CPT], z1[CPT];
        unit_load<CPT>(pr + e, here);
        unit_load<CPT>(pr + e - PXS, a);
        unit_load<CPT>(pr + e + PXS, b);
        unit_load<CPT>(sm.v[sp][NQ] + e, z0);
        unit_load<CPT>(sm.v[sn][NQ] + e, z1);
#pragma unroll
        for (int u = 0; u < CPT; u++) {
            ny_[u] = a[u] + b[u];
            nz_[u] = z0[u] + z1[u];
        }
    }
#pragma unroll
    for (int u = 0; u < CPT; u++)
        nx_[u] = (u == 0 ? pr[e - 1] : here[u - 1]) + (u == CPT - 1 ? pr[e + CPT] : here[u + 1]);

    // stage values and exchange fields of the unit's cells
    float m[CPT][NS][3], B[CPT][NS][3];
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = s * 3 + k;
            const float *vc = sm.v[sc][q], *vp = sm.v[sp][q], *vn = sm.v[sn][q];
            float cen[CPT], ya[CPT], yb[CPT], za[CPT], zb[CPT];
            unit_load<CPT>(vc + e, cen);
            unit_load<CPT>(vc + e - PXS, ya);
            unit_load<CPT>(vc + e + PXS, yb);
            unit_load<CPT>(vp + e, za);
            unit_load<CPT>(vn + e, zb);
            const float left = vc[e - 1], right = vc[e + CPT];
#pragma unroll
            for (int u = 0; u < CPT; u++) {
                const float xl = u == 0 ? left : cen[u - 1], xr = u == CPT - 1 ? right : cen[u + 1];
                m[u][s][k] = cen[u];
                // exchange: sum over present neighbours of (m_j - m_i) / c_d^2 (absent ones hold 0)
                B[u][s][k] = c.wx * (xl + xr - nx_[u] * cen[u]) +
                             c.wy * (ya[u] + yb[u] - ny_[u] * cen[u]) +
                             c.wz * (za[u] + zb[u] - nz_[u] * cen[u]);
            }
        }

    float kv[CPT][NS][3];
#pragma unroll
    for (int u = 0; u < CPT; u++) {
        float ucell[MAXN];
#pragma unroll
        for (int n = 0; n < MAXN; n++)
            ucell[n] = (HU && n < c.nmodes)
                           ? sm.upool[(size_t)(p % SM::D) * SM::USLOT + n * CW + oc + u] : 1.f;
        float bdem[3] = {0.f, 0.f, 0.f};
        if (c.fd && here[u] != 0.f)
#pragma unroll
            for (int k = 0; k < 3; k++) bdem[k] = __ldcg(c.bd + (size_t)k * c.ncell + idx + u);
        // a non-magnetic cell of the unit holds m = 0, so its overlap terms are exactly 0
        cell_slope<NS, HU>(c, cf, m[u], B[u], ucell, bdem, acc, kv[u]);
        if (here[u] == 0.f)
#pragma unroll
            for (int s = 0; s < NS; s++)
#pragma unroll
                for (int k = 0; k < 3; k++) kv[u][s][k] = 0.f;
    }

    // stores of the unit: one store per cell and component
    auto put = [&](float *base, int q, const float (&val)[CPT]) {
        float *dst = base + (size_t)q * c.ncell + idx;
#pragma unroll
        for (int u = 0; u < CPT; u++) dst[u] = val[u];
    };
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = s * 3 + k;
            float o[CPT];
#pragma unroll
            for (int u = 0; u < CPT; u++) o[u] = kv[u][s][k];
            put(kout, q, o);
            if (S >= 2 && rslot >= 0) {
#pragma unroll
                for (int u = 0; u < CPT; u++) o[u] = m[u][s][k];
                put(c.rec_m + ((size_t)rslot * 6 + (S >= 2 ? S - 2 : 0)) * NQ * c.ncell, q, o);
            }
        }
    if ((S == 1 || S == 7) && tslot >= 0) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            float r[CPT];
#pragma unroll
            for (int u = 0; u < CPT; u++) {
                const float *mm = m[u][s];
                r[u] = (S == 7 && here[u] != 0.f)
                           ? rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]) : 1.f;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                float om[CPT], ok[CPT];
#pragma unroll
                for (int u = 0; u < CPT; u++) {
                    om[u] = m[u][s][k] * r[u];
                    ok[u] = kv[u][s][k];
                }
                put(c.traj_m + (size_t)tslot * NQ * c.ncell, s * 3 + k, om);
                put(c.traj_k + (size_t)tslot * NQ * c.ncell, s * 3 + k, ok);
            }
        }
    }
    if (S >= 2 && S <= 6 && !c.stage_only) {
        // next stage value m_{S+1} = m_n + sum_j (h a_{S+1,j}) k_j, k_S last; error partial
#pragma unroll
        for (int s = 0; s < NS; s++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int q = s * 3 + k;
                float a[CPT], es[CPT];
                unit_load<CPT>(op + (0 * NQ + q) * CW + oc, a);
#pragma unroll
                for (int u = 0; u < CPT; u++) es[u] = 0.f;
#pragma unroll
                for (int o = 1; o < NO; o++) {
                    const int j = op_slope(S, o);
                    float kj[CPT];
                    unit_load<CPT>(op + (o * NQ + q) * CW + oc, kj);
#pragma unroll
                    for (int u = 0; u < CPT; u++) {
                        a[u] = fmaf(cf.cf[S][j], kj[u], a[u]);
                        if (S == 6) es[u] = fmaf(cf.e[j], kj[u], es[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < CPT; u++) {
                    a[u] = here[u] != 0.f ? fmaf(cf.cf[S][S - 1], kv[u][s][k], a[u]) : 0.f;
                    es[u] = here[u] != 0.f ? fmaf(cf.e[5], kv[u][s][k], es[u]) : 0.f;
                }
                const unsigned long long keep = l2_keep();
                st_hint(c.msv[(S + 1) & 1] + (size_t)q * c.ncell + idx, a[0], keep);
                if (S == 6) st_hint(c.es + (size_t)q * c.ncell + idx, es[0], keep);
            }
    }
    if (S == 7) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            float r[CPT];
#pragma unroll
            for (int u = 0; u < CPT; u++) {
                const float *mm = m[u][s];
                r[u] = here[u] != 0.f ? rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]) : 0.f;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int q = s * 3 + k;
                float o[CPT];
#pragma unroll
                for (int u = 0; u < CPT; u++) {
                    o[u] = m[u][s][k] * r[u];
                    if (here[u] != 0.f) {
                        const float e7 = cf.h * fmaf(cf.e[6], kv[u][s][k], op[q * CW + oc + u]);
                        acc.emax = nanmax(acc.emax, fabsf(e7));
                    }
                }
                put(mnew, q, o);
            }
        }
    }
}

// Start stage S's stream: row entries of the first planes and the first D planes of copies.
// Needs only m_n, the slopes of earlier stages and the stage values stored by the previous stage,
// so it can run before the cavity update of the previous stage is known.  Planes of the block's
// segments: segment t covers x in [x0, x0+CX), y in [y0, y0+WY), z in [z0, z1) and contributes
// planes z0-1 .. z1.
template <int NS, int CX, int WY, bool HU, int S>
__device__ void tiles_begin(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm, const float *mn,
                            Pipe &pp)
{
    using SM = StageSmem<NS, CX, WY, HU>;
    constexpr int D = SM::D, AHEAD = D + 1, PY = SM::PY, PXS = SM::PXS, CPT = SM::CPT;
    constexpr int OFF = SM::OFF;
    pp.gend = 0;
    for (int t = 0; t < sm.nseg; t++) pp.gend += sm.seg[t].w - sm.seg[t].z + 2;
    pp.nq = 0;
    if (sm.nseg == 0) return;
    const int i = threadIdx.x;
    pp.eo = (i / 32 + 1) * PXS + OFF + CPT * (i % 32);
    pp.er = -1;
    pp.rr = pp.rc = pp.rk = 0;
    // rim: threads 0..63 the units of rows 0 and PY-1, the next 2 PY the single cells of columns
    // OFF-1 and OFF+CX (the rim loads stay in as few warps as possible: a warp pays for its rim
    // loads whenever one of its lanes has one)
    if (i < SM::NRU) {
        pp.rk = 1;
        pp.rr = i < 32 ? 0 : PY - 1;
        pp.rc = CPT * (i % 32);
        pp.er = pp.rr * PXS + OFF + pp.rc;
    } else if (i < SM::NRU + SM::NRS) {
        const int j = i - SM::NRU;
        pp.rk = 2;
        pp.rr = j % PY;
        pp.rc = j < PY ? -1 : CX;
        pp.er = pp.rr * PXS + OFF + pp.rc;
    }
    pp.cr = cursor_start(sm);
    pp.ci = pp.cr;
    __syncthreads();   // the previous stage may still read the shared buffers
    for (int g = 0; g <= AHEAD; g++)
        if (i < PY && g < pp.gend) {
            cursor_seek(sm, pp.cr, g);
            sm.rows[g & 7][i] = g < ROWC ? sm.rowc[g][i]
                                         : row_entry(c, pp.cr.y0 - 1 + i, pp.cr.z0 - 1 + (g - pp.cr.off));
        }
    __syncthreads();
    for (; pp.nq < D; pp.nq++) {
        issue_tile<NS, CX, WY, HU, S>(c, sm, mn, pp.nq, pp);
        issue_ops<NS, CX, WY, HU, S>(c, sm, mn, pp.nq, pp);
    }
}

// Run stage S's stream to its end.  Commit groups come in the order tile(g), ops(g) for
// g = 0, 1, ...; at the start of iteration p the groups of planes up to p+D-1 are committed.
// Iteration p: wait for plane p+1's tile (and plane p's operands; stage 2: form plane p+1's tile
// values), publish it with the block barrier, issue plane p+D's tile, compute plane p, issue
// plane p+D's operands into the slot plane p has just released.  Only planes interior to their
// segment are computed.
template <int NS, int CX, int WY, bool HU, int S>
__device__ void tiles_run(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm, float *kout,
                          const float *mn, float *mnew, const Coef &cf, Pipe &pp, int tslot,
                          int rslot, Acc &acc)
{
    using SM = StageSmem<NS, CX, WY, HU>;
    constexpr int D = SM::D, AHEAD = D + 1, PY = SM::PY;
    constexpr int PEND = 2 * D - 3;   // groups after tile(p+1): ops(p+1), then D-2 planes
    static_assert(D >= 2, "two planes in flight at least");
    const int gend = pp.gend;
    if (sm.nseg == 0) return;
    const int i = threadIdx.x;
    auto load_rows = [&](int g) {   // rows of stream plane g into ring slot g mod 8
        if (i < PY && g < gend) {
            cursor_seek(sm, pp.cr, g);
            sm.rows[g & 7][i] = g < ROWC ? sm.rowc[g][i]
                                         : row_entry(c, pp.cr.y0 - 1 + i, pp.cr.z0 - 1 + (g - pp.cr.off));
        }
    };
    // planes 0 and 1 (committed: 0 .. D-1; plane 0 is a halo plane: its operand slot is free)
    cp_async_wait<PEND>();
    tile_combine<NS, CX, WY, HU, S>(c, sm, cf, 0, pp);
    tile_combine<NS, CX, WY, HU, S>(c, sm, cf, 1, pp);
    issue_tile<NS, CX, WY, HU, S>(c, sm, mn, pp.nq, pp);
    issue_ops<NS, CX, WY, HU, S>(c, sm, mn, pp.nq, pp);
    pp.nq++;
    for (int p = 1; p <= gend - 2; p++) {
        load_rows(p + AHEAD);
        cp_async_wait<PEND>();
        tile_combine<NS, CX, WY, HU, S>(c, sm, cf, p + 1, pp);
        __syncthreads();
        issue_tile<NS, CX, WY, HU, S>(c, sm, mn, pp.nq, pp);
        compute_cell<NS, CX, WY, HU, S>(c, sm, kout, mnew, cf, p, tslot, rslot, pp, acc);
        issue_ops<NS, CX, WY, HU, S>(c, sm, mn, pp.nq, pp);
        pp.nq++;
    }
    cp_async_wait<0>();
}

// Row-table entries of the first ROWC planes of the block's stream into the cache (once per
// launch, after the block's segments are known).
template <int NS, int CX, int WY, bool HU>
__device__ void stage_cache_rows(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm)
{
    using SM = StageSmem<NS, CX, WY, HU>;
    constexpr int PY = SM::PY;
    if (sm.nseg == 0) return;
    int gend = 0;
    for (int t = 0; t < sm.nseg; t++) gend += sm.seg[t].w - sm.seg[t].z + 2;
    const int n = (gend < ROWC ? gend : ROWC) * PY;
    for (int e = threadIdx.x; e < n; e += SM::NT) {
        const int g = e / PY, r = e - g * PY;
        Cursor cu = cursor_start(sm);
        cursor_seek(sm, cu, g);
        sm.rowc[g][r] = row_entry(c, cu.y0 - 1 + r, cu.z0 - 1 + (g - cu.off));
    }
}

// Engine-facing names of the stage code of this tile type (overloaded by smem type).
template <int S, int NS, int CX, int WY, bool HU>
__device__ __forceinline__ void stage_begin(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm,
                                            const float *mn, Pipe &pp)
{
    tiles_begin<NS, CX, WY, HU, S>(c, sm, mn, pp);
}

template <int S, int NS, int CX, int WY, bool HU>
__device__ __forceinline__ void stage_run(const Ctx &c, StageSmem<NS, CX, WY, HU> &sm,
                                          float *kout, const float *mn, float *mnew,
                                          const Coef &cf, Pipe &pp, int tslot, int rslot,
                                          Acc &acc)
{
    tiles_run<NS, CX, WY, HU, S>(c, sm, kout, mn, mnew, cf, pp, tslot, rslot, acc);
}

// Magnetic cells a thread of this tile type computes per plane (the overlap sums' bound).
template <int NS, int CX, int WY, bool HU>
__host__ __device__ constexpr int cells_per_thread(const StageSmem<NS, CX, WY, HU> *)
{
    return CX / 32;
}

}  // namespace cmx
