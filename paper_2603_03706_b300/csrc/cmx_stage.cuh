// Device code of one Dormand-Prince stage over the tiles of a masked grid (sm_103a).
//
// One stage S computes, for every magnetic cell,
//   m_S  = m_n + h sum_{j<S} a_Sj k_j                      (stage combination, FP32)
//   B    = exchange(m_S) + anisotropy + Zeeman + demag + inter-sublattice + B_rf(a_S)
//   k_S  = -gamma/(1+alpha^2) [ m_S x B + alpha m_S x (m_S x B) ]      (LLG, Sec. II A)
// and the block partial sums of the overlaps u_n (m_x - i m_y) (Eq. (18)).  Stage 7 also
// writes the renormalised 5th-order point and the block maximum of |e_m|,
// e_m = h sum_j E_j k_j.
//
// Tiles are columns of (WX-2) x (WY-2) cells, several planes deep; a block of WX x WY threads
// covers a tile with its one-cell halo rim and marches through it plane by plane.  The raw
// operands of the next planes arrive by asynchronous copies (cp.async) into shared memory while
// the block combines the oldest plane into a ring of four planes of stage values and computes
// the plane before it from planes p-1, p, p+1: one __syncthreads per plane, the 6-neighbour
// stencil reads only shared memory.  Cells are stored compactly per (y, z) row between the first
// and the last magnetic x of the row; the row table gives the offset.
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

// Slopes read by stage S (1-based): those with a nonzero coupling, and at stage 7 also those
// with a nonzero error weight.  Array 0 of a stage is m_n, arrays 1.. are these slopes.
__host__ __device__ constexpr bool slope_used(int S, int j)
{
    return j < S - 1 && (dp_a(S - 1, j) != 0.0 || (S == 7 && dp_e(j) != 0.0));
}

__host__ __device__ constexpr int n_arrays(int S)
{
    int n = 1;
    for (int j = 0; j < 6; j++) n += slope_used(S, j) ? 1 : 0;
    return n;
}

__host__ __device__ constexpr int array_slope(int S, int a)
{
    int n = 0;
    for (int j = 0; j < 6; j++)
        if (slope_used(S, j)) {
            n++;
            if (n == a) return j;
        }
    return -1;
}

// Compensated FP32 pair ("double-float"): value = hi + lo, about 44 significant bits.  Used for
// the overlap sums across threads and blocks; FP64 has a long dependent latency on this part.
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

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
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

// Shared memory of a block whose threads cover a WX x WY window: the interior
// (WX-2) x (WY-2) cells are computed, the one-cell rim is the halo.  D planes of raw operands
// (m_n and the slopes of the stage) are in flight as asynchronous copies while the block
// combines the oldest one into the ring of stage values and computes the plane before it.
template <int NS, int WX, int WY, bool HU>
struct StageSmem {
    static constexpr int W = WX * WY;
    static constexpr int NQ = NS * 3;
    static constexpr int RING = 4;
    static constexpr int NAMAX = 6;             // m_n + at most five slopes per stage
    static constexpr int POOL = (NS == 1 ? 2 : 1) * NAMAX * NQ * W;   // raw operand floats
    static constexpr int DMAX = 4;
    // Planes in flight at stage S: as many plane slots of n_arrays(S) x NQ x W floats as the
    // pool holds (at most 4).
    template <int S>
    __host__ __device__ static constexpr int depth()
    {
        const int d = POOL / (n_arrays(S) * NQ * W);
        return d < 1 ? 1 : (d > DMAX ? DMAX : d);
    }
    float raw[POOL];              // raw operands of planes in flight, [slot][array][q][W]
    int ridx[DMAX][W];            // their compact indices (-1: absent)
    float v[RING][NQ + 1][W];     // stage values and presence (last row) of four planes
    float es[2][NQ][W];           // stage 7: sum_{j<7} E_j k_j of the interior cells
    int cidx[2][W];               // compact index of the interior cells (-1: absent)
    F2 red[32][2 * MAXN];         // per-warp partial overlaps
    float redmax[32];
    const float *kp[7];           // physical slope buffers in logical order
    int2 rows[8][WY];             // row-table entries of the window rows, by plane mod 8
    int2 rowc[ROWC][WY];          // the same for the first ROWC planes of the stream (every
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

// Compact index of box cell x in a row given its row-table entry, or -1.
__device__ __forceinline__ int row_index(const Ctx &c, int2 r, int x)
{
    const int xs = r.y & 0xffff, xe = (int)((unsigned)r.y >> 16);
    if (x < xs || x >= xe) return -1;
    const int idx = r.x + (x - xs);
    if (c.active && !((__ldg(&c.active[idx >> 5]) >> (idx & 31)) & 1u)) return -1;
    return idx;
}

__device__ __forceinline__ int2 row_entry(const Ctx &c, int y, int z)
{
    if ((unsigned)y >= (unsigned)c.ny || (unsigned)z >= (unsigned)c.nz) return make_int2(0, 0);
    return __ldg(&c.rows[z * c.ny + y]);
}

// Issue the asynchronous copies of this thread's window position in stream plane g, then
// commit one copy group (possibly empty).
template <int NS, int WX, int WY, bool HU, int S>
__device__ __forceinline__ void issue_plane(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm,
                                            const float *mn, int g, int gend, const Cursor &cu,
                                            int r, int col, bool corner, bool inner_pos)
{
    using SM = StageSmem<NS, WX, WY, HU>;
    constexpr int NQ = NS * 3, NA = n_arrays(S), D = SM::template depth<S>();
    constexpr int W = SM::W;
    const int i = threadIdx.x;
    if (g < gend) {
        const int slot = g % D;
        float *rp = sm.raw + (size_t)slot * NA * NQ * W;
        const int idx = corner ? -1 : row_index(c, sm.rows[g & 7][r], cu.x0 - 1 + col);
        sm.ridx[slot][i] = idx;
        if (idx >= 0) {
#pragma unroll
            for (int k = 0; k < NQ; k++) {
                const size_t o = (size_t)k * c.ncell + idx;
                cp_async4(rp + (0 * NQ + k) * W + i, mn + o);
#pragma unroll
                for (int a = 1; a < NA; a++)
                    cp_async4(rp + (a * NQ + k) * W + i, sm.kp[array_slope(S, a)] + o);
            }
        }
    }
    cp_async_commit();
}

// Combine the raw operands of stream plane g (copied by this thread) into the stage value
// m_S = m_n + sum_j (h a_Sj) k_j, and at stage 7 the partial error sum of interior cells.
template <int NS, int WX, int WY, bool HU, int S>
__device__ __forceinline__ void combine_plane(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm,
                                              const Coef &cf, int g, bool inner_cell)
{
    using SM = StageSmem<NS, WX, WY, HU>;
    constexpr int NQ = NS * 3, NA = n_arrays(S), D = SM::template depth<S>();
    constexpr int R = SM::RING, W = SM::W;
    const int i = threadIdx.x;
    const int rs = g % D, vs = g % R;
    const float *rp = sm.raw + (size_t)rs * NA * NQ * W;
    const int idx = sm.ridx[rs][i];
    const bool here = idx >= 0;
#pragma unroll
    for (int k = 0; k < NQ; k++) {
        float acc = 0.f, es = 0.f;
        if (here) {
            acc = rp[(0 * NQ + k) * W + i];
#pragma unroll
            for (int a = 1; a < NA; a++) {
                const int j = array_slope(S, a);
                const float kj = rp[(a * NQ + k) * W + i];
                if (dp_a(S - 1, j) != 0.0) acc = fmaf(cf.cf[S - 1][j], kj, acc);
                if (S == 7 && dp_e(j) != 0.0) es = fmaf(cf.e[j], kj, es);
            }
        }
        sm.v[vs][k][i] = acc;
        if (S == 7 && inner_cell) sm.es[g & 1][k][i] = es;
    }
    sm.v[vs][NQ][i] = here ? 1.f : 0.f;
    sm.cidx[g & 1][i] = (inner_cell && here) ? idx : -1;
}

// RHS of this thread's interior cell of plane p (ring slots: p-1, p, p+1).  Writes k_S (and at
// stage 7 the renormalised new m) and accumulates the overlap sums and the error maximum.
template <int NS, int WX, int WY, bool HU, int S>
__device__ __forceinline__ void compute_cell(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm,
                                             float *kout, float *mnew, const Coef &cf, int p,
                                             const float *ucell, int tslot, int rslot,
                                             Acc &acc)
{
    using SM = StageSmem<NS, WX, WY, HU>;
    constexpr int NQ = SM::NQ, R = SM::RING;
    const int i = threadIdx.x;
    const int idx = sm.cidx[p & 1][i];
    if (idx < 0) return;
    const int sp = (p + R - 1) % R, sc = p % R, sn = (p + 1) % R;

    const float nx_ = sm.v[sc][NQ][i - 1] + sm.v[sc][NQ][i + 1];
    const float ny_ = sm.v[sc][NQ][i - WX] + sm.v[sc][NQ][i + WX];
    const float nz_ = sm.v[sp][NQ][i] + sm.v[sn][NQ][i];

    float m[NS][3], B[NS][3];
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int q = s * 3 + k;
            const float cen = sm.v[sc][q][i];
            m[s][k] = cen;
            // exchange: sum over present neighbours of (m_j - m_i) / c_d^2 (absent ones hold 0)
            B[s][k] = c.wx * (sm.v[sc][q][i - 1] + sm.v[sc][q][i + 1] - nx_ * cen) +
                      c.wy * (sm.v[sc][q][i - WX] + sm.v[sc][q][i + WX] - ny_ * cen) +
                      c.wz * (sm.v[sp][q][i] + sm.v[sn][q][i] - nz_ * cen);
        }

    float mt[3];
#pragma unroll
    for (int k = 0; k < 3; k++) mt[k] = (NS == 2) ? (m[0][k] + m[1][k]) : m[0][k];
    // feedback field sum_n u_n (2/gamma) Re[g~_n a_n] and the overlap partial sums of the net
    // moment (m1 + m2)/2 with the same profile values
    const float hx = (NS == 2) ? 0.5f * mt[0] : mt[0];
    const float hy = (NS == 2) ? 0.5f * mt[1] : mt[1];
    float brf = 0.f;
#pragma unroll
    for (int n = 0; n < MAXN; n++) {
        if (n < c.nmodes) {
            const float un = HU ? ucell[n] : 1.f;
            brf = fmaf(un, cf.hrf[n], brf);
            acc.re[n] = fmaf(un, hx, acc.re[n]);
            acc.im[n] = fmaf(-un, hy, acc.im[n]);
        }
    }

#pragma unroll
    for (int s = 0; s < NS; s++) {
        const float mk = m[s][0] * c.ku[0] + m[s][1] * c.ku[1] + m[s][2] * c.ku[2];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float b = B[s][k] + c.anis * mk * c.ku[k] + c.B0[k] - c.dmg[k] * mt[k];
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
        const float kv[3] = {c.pre * fmaf(c.alpha, t2x, t1x), c.pre * fmaf(c.alpha, t2y, t1y),
                             c.pre * fmaf(c.alpha, t2z, t1z)};
#pragma unroll
        for (int k = 0; k < 3; k++) kout[(size_t)(s * 3 + k) * c.ncell + idx] = kv[k];
        if (S >= 2 && rslot >= 0) {
            const size_t o = ((size_t)rslot * 6 + (S >= 2 ? S - 2 : 0)) * NQ * c.ncell;
#pragma unroll
            for (int k = 0; k < 3; k++) c.rec_m[o + (size_t)(s * 3 + k) * c.ncell + idx] = mm[k];
        }
        if ((S == 1 || S == 7) && tslot >= 0) {
            const size_t o = (size_t)tslot * NQ * c.ncell;
            const float r = S == 7 ? rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]) : 1.f;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                c.traj_m[o + (size_t)(s * 3 + k) * c.ncell + idx] = mm[k] * r;
                c.traj_k[o + (size_t)(s * 3 + k) * c.ncell + idx] = kv[k];
            }
        }
        if (S == 7) {
            const float r = rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int q = s * 3 + k;
                mnew[(size_t)q * c.ncell + idx] = mm[k] * r;
                const float e = cf.h * fmaf(cf.e[6], kv[k], sm.es[p & 1][q][i]);
                acc.emax = nanmax(acc.emax, fabsf(e));
            }
        }
    }
}

// Copy-pipeline state of one stage: cursors for row loading (cr), copy issue (ci) and combine
// (cc), the next plane to issue and the stream length.
struct Pipe {
    Cursor cr, ci, cc;
    int nq, gend;
    int fidx, fnib, finner;   // quad windows: the first plane, issued by stage_begin
};

// Start stage S's stream: row entries of the first planes and the first D planes of copies.
// Needs only m_n and the slopes of earlier stages, so it can run before the cavity update of
// the previous stage is known.  Planes of the block's segments: segment t covers interior x in
// [x0, x0+WX-2), y in [y0, y0+WY-2), z in [z0, z1) and contributes planes z0-1 .. z1.
template <int NS, int WX, int WY, bool HU, int S>
__device__ void tiles_begin(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm, const float *mn,
                            Pipe &pp)
{
    constexpr int D = StageSmem<NS, WX, WY, HU>::template depth<S>();
    constexpr int AHEAD = D + 3;   // row entries are loaded this many planes ahead (ring of 8)
    pp.gend = 0;
    for (int t = 0; t < sm.nseg; t++) pp.gend += sm.seg[t].w - sm.seg[t].z + 2;
    pp.nq = 0;
    if (sm.nseg == 0) return;
    const int r = threadIdx.x / WX, col = threadIdx.x - (threadIdx.x / WX) * WX;
    const bool corner = (r == 0 || r == WY - 1) && (col == 0 || col == WX - 1);
    const bool inner_pos = r >= 1 && r <= WY - 2 && col >= 1 && col <= WX - 2;
    pp.cr = cursor_start(sm);
    pp.ci = pp.cr;
    pp.cc = pp.cr;
    __syncthreads();   // the previous stage may still read the shared buffers
    for (int g = 0; g <= AHEAD; g++)
        if (threadIdx.x < WY && g < pp.gend) {
            cursor_seek(sm, pp.cr, g);
            sm.rows[g & 7][threadIdx.x] =
                g < ROWC ? sm.rowc[g][threadIdx.x]
                         : row_entry(c, pp.cr.y0 - 1 + threadIdx.x, pp.cr.z0 - 1 + (g - pp.cr.off));
        }
    __syncthreads();
    for (; pp.nq < D; pp.nq++) {
        cursor_seek(sm, pp.ci, pp.nq);
        issue_plane<NS, WX, WY, HU, S>(c, sm, mn, pp.nq, pp.gend, pp.ci, r, col, corner,
                                       inner_pos);
    }
}

// Run stage S's stream to its end: combine the oldest plane in flight, issue the next, compute
// the plane before it.  Only planes interior to their segment are computed; the profiles of
// the next computed cell are loaded one plane ahead.
template <int NS, int WX, int WY, bool HU, int S>
__device__ void tiles_run(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm, float *kout,
                          const float *mn, float *mnew, const Coef &cf, Pipe &pp, int tslot,
                          int rslot, Acc &acc)
{
    constexpr int D = StageSmem<NS, WX, WY, HU>::template depth<S>();
    constexpr int AHEAD = D + 3;
    const int gend = pp.gend;
    if (sm.nseg == 0) return;
    const int r = threadIdx.x / WX, col = threadIdx.x - (threadIdx.x / WX) * WX;
    const bool corner = (r == 0 || r == WY - 1) && (col == 0 || col == WX - 1);
    const bool inner_pos = r >= 1 && r <= WY - 2 && col >= 1 && col <= WX - 2;
    auto load_rows = [&](int g) {   // rows of stream plane g into ring slot g mod 8
        if (threadIdx.x < WY && g < gend) {
            cursor_seek(sm, pp.cr, g);
            sm.rows[g & 7][threadIdx.x] =
                g < ROWC ? sm.rowc[g][threadIdx.x]
                         : row_entry(c, pp.cr.y0 - 1 + threadIdx.x, pp.cr.z0 - 1 + (g - pp.cr.off));
        }
    };
    auto inner_at = [&](const Cursor &cu, int g) {
        const int q = g - cu.off;
        return inner_pos && q >= 1 && q <= cu.np - 2;
    };
    float ucur[MAXN], unext[MAXN];
#pragma unroll
    for (int n = 0; n < MAXN; n++) ucur[n] = unext[n] = 1.f;
    auto load_u = [&](int g, float *dst) {   // profiles of this thread's cell of plane g
        if (!HU) return;
        const int idx = sm.cidx[g & 1][threadIdx.x];
#pragma unroll
        for (int n = 0; n < MAXN; n++)
            if (n < c.nmodes && idx >= 0) dst[n] = __ldg(c.u + (size_t)n * c.ncell + idx);
    };
    for (int g = 0; g < 2 && g < gend; g++) {
        cp_async_wait<D - 1>();
        cursor_seek(sm, pp.cc, g);
        combine_plane<NS, WX, WY, HU, S>(c, sm, cf, g, inner_at(pp.cc, g));
        cursor_seek(sm, pp.ci, pp.nq);
        issue_plane<NS, WX, WY, HU, S>(c, sm, mn, pp.nq, gend, pp.ci, r, col, corner,
                                       inner_pos);
        pp.nq++;
    }
    load_u(1, unext);
    for (int p = 1; p <= gend - 2; p++) {
        load_rows(p + AHEAD);
        // plane p+1: its copies are the oldest in flight
        cp_async_wait<D - 1>();
        cursor_seek(sm, pp.cc, p + 1);
        combine_plane<NS, WX, WY, HU, S>(c, sm, cf, p + 1, inner_at(pp.cc, p + 1));
        cursor_seek(sm, pp.ci, pp.nq);
        issue_plane<NS, WX, WY, HU, S>(c, sm, mn, pp.nq, gend, pp.ci, r, col, corner,
                                       inner_pos);
        pp.nq++;
#pragma unroll
        for (int n = 0; n < MAXN; n++) ucur[n] = unext[n];
        load_u(p + 1, unext);
        __syncthreads();
        compute_cell<NS, WX, WY, HU, S>(c, sm, kout, mnew, cf, p, ucur, tslot, rslot, acc);
    }
    cp_async_wait<0>();
}

// Row-table entries of the first ROWC planes of the block's stream into the cache (once per
// launch, after the block's segments are known).
template <int NS, int WX, int WY, bool HU>
__device__ void stage_cache_rows(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm)
{
    if (sm.nseg == 0) return;
    int gend = 0;
    for (int t = 0; t < sm.nseg; t++) gend += sm.seg[t].w - sm.seg[t].z + 2;
    const int n = (gend < ROWC ? gend : ROWC) * WY;
    for (int e = threadIdx.x; e < n; e += WX * WY) {
        const int g = e / WY, r = e - g * WY;
        Cursor cu = cursor_start(sm);
        cursor_seek(sm, cu, g);
        sm.rowc[g][r] = row_entry(c, cu.y0 - 1 + r, cu.z0 - 1 + (g - cu.off));
    }
}

// Engine-facing names of the stage code of this window type (overloaded by smem type).
template <int S, int NS, int WX, int WY, bool HU>
__device__ __forceinline__ void stage_begin(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm,
                                            const float *mn, Pipe &pp)
{
    tiles_begin<NS, WX, WY, HU, S>(c, sm, mn, pp);
}

template <int S, int NS, int WX, int WY, bool HU>
__device__ __forceinline__ void stage_run(const Ctx &c, StageSmem<NS, WX, WY, HU> &sm,
                                          float *kout, const float *mn, float *mnew,
                                          const Coef &cf, Pipe &pp, int tslot, int rslot,
                                          Acc &acc)
{
    tiles_run<NS, WX, WY, HU, S>(c, sm, kout, mn, mnew, cf, pp, tslot, rslot, acc);
}

}  // namespace cmx
