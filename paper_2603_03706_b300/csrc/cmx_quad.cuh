// Stage code with four consecutive x-cells per thread ("quads"), one sublattice (sm_103a).
//
// The same stage as cmx_stage.cuh (combination, fields, torque, overlaps, error; see there),
// laid out for 16-byte memory operations: rows are stored on 4-cell boundaries (the layout is
// built with align = 4, padding cells inactive), so each thread loads its quad of every operand
// with one 16-byte load per component, combines it in registers and stores its slopes with
// 16-byte stores.  A WQ x WY thread window covers (WQ-2) x (WY-2) interior quads plus a one-quad
// rim; only the rim quads' adjacent cells are used by the stencil.  Along z the thread keeps the
// stage values of its quad for planes p-1, p, p+1 in registers, so the z-neighbours cost no
// shared-memory traffic; x- and y-neighbours come from a three-plane ring in shared memory.  The
// loads of plane p+2 are issued (into registers) before plane p is computed, one __syncthreads
// per plane.
#pragma once

#include "cmx_stage.cuh"

namespace cmx {

constexpr int QMAX_NT = 256;    // threads of a quad window (WQ x WY, a multiple of 32)
constexpr int QMAX_WY = 16;

// Fixed part of the quad kernel's shared memory (the engine-facing members) followed by the
// window-sized rings: stage values, presence nibbles, stage-7 error partials, profiles.
struct QuadHead {
    F2 red[32][2 * MAXN];
    float redmax[32];
    const float *kp[7];
    int2 rows[8][QMAX_WY];
    int4 seg[MAX_BLOCK_SEGMENTS];
    int nseg;
};

__host__ __device__ constexpr size_t quad_head_bytes()
{
    return (sizeof(QuadHead) + 15) / 16 * 16;
}

// Shared-memory bytes of a quad window of nt threads with nu profiled modes.
__host__ __device__ constexpr size_t quad_smem_bytes(int nt, int nu)
{
    return quad_head_bytes() + (size_t)nt * 16 * (6 * 3     // raw operands of one plane
                                                  + 3 * 3    // stage values, 3 planes
                                                  + 2 * 3    // stage 7 partial errors, 2 planes
                                                  + 3 * nu)  // profiles, 3 planes
           + (size_t)3 * nt;                                 // presence nibbles
}

template <bool HU>
struct QuadSmem {
    F2 (*red)[2 * MAXN];
    float *redmax;
    const float **kp;
    int2 (*rows)[QMAX_WY];
    int4 *seg;
    int &nseg;
    int wq, wy, nt, nu;
    float4 *raw;         // [6][3][nt] this thread's raw operands of the plane in flight
    float4 *sv;          // [3][3][nt] stage values of the window, ring of three planes
    float4 *es;          // [2][3][nt] stage 7: sum_{j<7} E_j k_j of this thread's quad
    float4 *us;          // [3][nu][nt] profiles of this thread's quad, ring of three planes
    unsigned char *pr;   // [3][nt] presence nibble of each quad
};

template <bool HU>
__device__ __forceinline__ QuadSmem<HU> quad_smem(unsigned char *raw, int wq, int wy, int nmodes)
{
    QuadHead &h = *reinterpret_cast<QuadHead *>(raw);
    const int nt = wq * wy, nu = HU ? nmodes : 0;
    float4 *t = reinterpret_cast<float4 *>(raw + quad_head_bytes());
    float4 *rp = t;
    float4 *sv = rp + 18 * nt;
    float4 *es = sv + 9 * nt;
    float4 *us = es + 6 * nt;
    unsigned char *pr = reinterpret_cast<unsigned char *>(us + 3 * nu * nt);
    return QuadSmem<HU>{h.red, h.redmax, h.kp, h.rows, h.seg, h.nseg, wq, wy, nt, nu,
                        rp, sv, es, us, pr};
}

__device__ __forceinline__ float f4get(const float4 &v, int c)
{
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

__device__ __forceinline__ void f4set(float4 &v, int c, float x)
{
    if (c == 0) v.x = x;
    else if (c == 1) v.y = x;
    else if (c == 2) v.z = x;
    else v.w = x;
}

__device__ __forceinline__ float4 f4fma(float a, const float4 &b, const float4 &c)
{
    return make_float4(fmaf(a, b.x, c.x), fmaf(a, b.y, c.y), fmaf(a, b.z, c.z),
                       fmaf(a, b.w, c.w));
}

__device__ __forceinline__ float4 f4mask(const float4 &v, unsigned nib)
{
    return make_float4((nib & 1u) ? v.x : 0.f, (nib & 2u) ? v.y : 0.f, (nib & 4u) ? v.z : 0.f,
                       (nib & 8u) ? v.w : 0.f);
}

// The plane in flight for this thread's quad (its operands are in sm.raw).
struct QuadRaw {
    int idx;              // compact index of the quad's first cell, or -1
    unsigned nib;         // presence of its four cells
    bool inner;           // the quad is computed (interior position, interior plane)
};

// Issue the 16-byte asynchronous copies of plane g for this thread's quad: m_n and the slopes
// of stage S into sm.raw, the profiles (computed quads only) into the profile ring.
template <int S, bool HU>
__device__ __forceinline__ void quad_issue(const Ctx &c, QuadSmem<HU> &sm, const float *mn, int g,
                                           int gend, Cursor &cu, int r, int qx, bool corner,
                                           bool inner_pos, QuadRaw &rw)
{
    constexpr int NA = n_arrays(S);
    rw.idx = -1;
    rw.nib = 0;
    rw.inner = false;
    if (g >= gend) return;
    cursor_seek(sm, cu, g);
    const int q = g - cu.off;
    rw.inner = inner_pos && q >= 1 && q <= cu.np - 2;
    if (corner) return;
    const int2 re = sm.rows[g & 7][r];
    const int xs = re.y & 0xffff, xe = (int)((unsigned)re.y >> 16);
    const int X = cu.x0 - 4 + 4 * qx;      // box x of the quad (multiple of 4, like xs and xe)
    if (X < xs || X >= xe) return;
    const int idx = re.x + (X - xs);
    rw.idx = idx;
    rw.nib = c.active ? (__ldg(&c.active[idx >> 5]) >> (idx & 31)) & 0xFu : 0xFu;
    const size_t n = (size_t)c.ncell;
    float4 *dst = sm.raw + threadIdx.x;
    const int nt = sm.nt;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        cp_async16(dst + (size_t)k * nt, mn + k * n + idx);
#pragma unroll
        for (int a = 1; a < NA; a++)
            cp_async16(dst + (size_t)(a * 3 + k) * nt, sm.kp[array_slope(S, a)] + k * n + idx);
    }
    if (HU && rw.inner) {
        float4 *dst = sm.us + (size_t)(g % 3) * sm.nu * sm.nt + threadIdx.x;
#pragma unroll
        for (int u = 0; u < MAXN; u++)
            if (u < c.nmodes) cp_async16(dst + (size_t)u * sm.nt, c.u + u * n + idx);
    }
}

// Centre quad of plane p: k_S of its present cells (16-byte stores), stage 7 the renormalised
// point and the error, the overlap partial sums; the adjoint stores when requested.
template <int S, bool HU>
__device__ __forceinline__ void quad_cell(const Ctx &c, QuadSmem<HU> &sm, float *kout,
                                          float *mnew, const Coef &cf, int p, const float4 *Vm,
                                          const float4 *V0, const float4 *Vp, unsigned nm,
                                          unsigned n0, unsigned np_, int idx, int tslot,
                                          int rslot, Acc &acc)
{
    const int i = threadIdx.x, nt = sm.nt, wq = sm.wq;
    const int sc = p % 3;
    const float4 *sv = sm.sv + (size_t)sc * 3 * nt;
    const unsigned char *pr = sm.pr + (size_t)sc * nt;
    const unsigned nl = pr[i - 1], nr = pr[i + 1], nd = pr[i - wq], nu = pr[i + wq];
    const size_t n = (size_t)c.ncell;
    const float4 *us = sm.us + (size_t)(p % 3) * sm.nu * nt + i;
    const float4 *es = sm.es + (size_t)(p & 1) * 3 * nt + i;
    float4 K[3], M[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        K[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        M[k] = K[k];
    }
#pragma unroll
    for (int cc = 0; cc < 4; cc++) {
        if (!((n0 >> cc) & 1u)) continue;
        // neighbour presence: x within the quad or the adjacent quads' edge cells
        const float pxm = cc > 0 ? (float)((n0 >> (cc - 1)) & 1u) : (float)((nl >> 3) & 1u);
        const float pxp = cc < 3 ? (float)((n0 >> (cc + 1)) & 1u) : (float)(nr & 1u);
        const float pym = (float)((nd >> cc) & 1u), pyp = (float)((nu >> cc) & 1u);
        const float pzm = (float)((nm >> cc) & 1u), pzp = (float)((np_ >> cc) & 1u);
        float m[3], B[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float cen = f4get(V0[k], cc);
            const float xm = cc > 0 ? f4get(V0[k], cc - 1) : sv[(size_t)k * nt + i - 1].w;
            const float xp = cc < 3 ? f4get(V0[k], cc + 1) : sv[(size_t)k * nt + i + 1].x;
            const float ym = f4get(sv[(size_t)k * nt + i - wq], cc);
            const float yp = f4get(sv[(size_t)k * nt + i + wq], cc);
            const float zm = f4get(Vm[k], cc), zp = f4get(Vp[k], cc);
            m[k] = cen;
            // absent neighbours hold 0 and count 0
            B[k] = c.wx * (xm + xp - (pxm + pxp) * cen) + c.wy * (ym + yp - (pym + pyp) * cen) +
                   c.wz * (zm + zp - (pzm + pzp) * cen);
        }
        float brf = 0.f;
#pragma unroll
        for (int u = 0; u < MAXN; u++)
            if (u < c.nmodes) {
                const float un = HU ? f4get(us[(size_t)u * nt], cc) : 1.f;
                brf = fmaf(un, cf.hrf[u], brf);
                acc.re[u] = fmaf(un, m[0], acc.re[u]);
                acc.im[u] = fmaf(-un, m[1], acc.im[u]);
            }
        const float mk = m[0] * c.ku[0] + m[1] * c.ku[1] + m[2] * c.ku[2];
#pragma unroll
        for (int k = 0; k < 3; k++) B[k] += c.anis * mk * c.ku[k] + c.B0[k] - c.dmg[k] * m[k];
        B[0] += brf;
        const float t1x = m[1] * B[2] - m[2] * B[1];
        const float t1y = m[2] * B[0] - m[0] * B[2];
        const float t1z = m[0] * B[1] - m[1] * B[0];
        const float t2x = m[1] * t1z - m[2] * t1y;
        const float t2y = m[2] * t1x - m[0] * t1z;
        const float t2z = m[0] * t1y - m[1] * t1x;
        const float kv[3] = {c.pre * fmaf(c.alpha, t2x, t1x), c.pre * fmaf(c.alpha, t2y, t1y),
                             c.pre * fmaf(c.alpha, t2z, t1z)};
#pragma unroll
        for (int k = 0; k < 3; k++) f4set(K[k], cc, kv[k]);
        if (S == 7) {
            const float rn = rsqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                f4set(M[k], cc, m[k] * rn);
                const float e = cf.h * fmaf(cf.e[6], kv[k], f4get(es[(size_t)k * nt], cc));
                acc.emax = nanmax(acc.emax, fabsf(e));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        reinterpret_cast<float4 *>(kout + k * n + idx)[0] = K[k];
        if (S == 7) reinterpret_cast<float4 *>(mnew + k * n + idx)[0] = M[k];
    }
    if (S >= 2 && rslot >= 0) {
        const size_t o = ((size_t)rslot * 6 + (S >= 2 ? S - 2 : 0)) * 3 * n;
#pragma unroll
        for (int k = 0; k < 3; k++)
            reinterpret_cast<float4 *>(c.rec_m + o + k * n + idx)[0] = f4mask(V0[k], n0);
    }
    if ((S == 1 || S == 7) && tslot >= 0) {
        const size_t o = (size_t)tslot * 3 * n;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            reinterpret_cast<float4 *>(c.traj_m + o + k * n + idx)[0] =
                S == 7 ? M[k] : f4mask(V0[k], n0);
            reinterpret_cast<float4 *>(c.traj_k + o + k * n + idx)[0] = K[k];
        }
    }
}

// Quad windows read their row entries from the table (no cache).
template <bool HU>
__device__ __forceinline__ void stage_cache_rows(const Ctx &, QuadSmem<HU> &)
{
}

// Start of stage S: the row entries of the first planes and an L2 prefetch of the first plane
// of the block's stream (the loads themselves are issued by stage_run).
template <int S, bool HU>
__device__ void stage_begin(const Ctx &c, QuadSmem<HU> &sm, const float *mn, Pipe &pp)
{
    constexpr int AHEAD = 4;
    pp.gend = 0;
    for (int t = 0; t < sm.nseg; t++) pp.gend += sm.seg[t].w - sm.seg[t].z + 2;
    pp.nq = 0;
    if (sm.nseg == 0) return;
    pp.cr = cursor_start(sm);
    pp.ci = pp.cr;
    pp.cc = pp.cr;
    __syncthreads();   // the previous stage may still read the shared buffers
    for (int g = 0; g <= AHEAD; g++)
        if ((int)threadIdx.x < sm.wy && g < pp.gend) {
            cursor_seek(sm, pp.cr, g);
            sm.rows[g & 7][threadIdx.x] =
                row_entry(c, pp.cr.y0 - 1 + threadIdx.x, pp.cr.z0 - 1 + (g - pp.cr.off));
        }
    __syncthreads();
    // the copies of the first plane (a halo plane) start before the cavity update of the
    // previous stage is known
    const int i = threadIdx.x, wq = sm.wq, wy = sm.wy;
    const int r = i / wq, qx = i - (i / wq) * wq;
    const bool corner = (r == 0 || r == wy - 1) && (qx == 0 || qx == wq - 1);
    const bool inner_pos = r >= 1 && r <= wy - 2 && qx >= 1 && qx <= wq - 2;
    QuadRaw rw;
    quad_issue<S, HU>(c, sm, mn, 0, pp.gend, pp.ci, r, qx, corner, inner_pos, rw);
    cp_async_commit();
    pp.fidx = rw.idx;
    pp.fnib = (int)rw.nib;
    pp.finner = rw.inner ? 1 : 0;
}

// Run stage S over the block's stream of planes.
template <int S, bool HU>
__device__ void stage_run(const Ctx &c, QuadSmem<HU> &sm, float *kout, const float *mn,
                          float *mnew, const Coef &cf, Pipe &pp, int tslot, int rslot, Acc &acc)
{
    constexpr int NA = n_arrays(S), AHEAD = 4;
    const int gend = pp.gend;
    if (sm.nseg == 0) return;
    const int i = threadIdx.x, nt = sm.nt, wq = sm.wq, wy = sm.wy;
    const int r = i / wq, qx = i - (i / wq) * wq;
    const bool corner = (r == 0 || r == wy - 1) && (qx == 0 || qx == wq - 1);
    const bool inner_pos = r >= 1 && r <= wy - 2 && qx >= 1 && qx <= wq - 2;
    auto load_rows = [&](int g) {
        if (i < wy && g < gend) {
            cursor_seek(sm, pp.cr, g);
            sm.rows[g & 7][i] = row_entry(c, pp.cr.y0 - 1 + i, pp.cr.z0 - 1 + (g - pp.cr.off));
        }
    };
    // combine the raw operands of plane g (this thread's copies in sm.raw) into its quad
    // (registers V, presence), publish it to the ring and, at stage 7, keep the partial error
    auto combine = [&](int g, const QuadRaw &rw, float4 *V, unsigned &nib, int &idx,
                       bool &inner) {
        const int vs = g % 3;
        nib = rw.idx >= 0 ? rw.nib : 0u;
        idx = rw.idx;
        inner = rw.inner && rw.idx >= 0 && nib != 0u;
        const float4 *src = sm.raw + i;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float4 acc4 = make_float4(0.f, 0.f, 0.f, 0.f), e4 = acc4;
            if (rw.idx >= 0) {
                acc4 = src[(size_t)k * nt];
#pragma unroll
                for (int a = 1; a < NA; a++) {
                    const int j = array_slope(S, a);
                    const float4 kj = src[(size_t)(a * 3 + k) * nt];
                    if (dp_a(S - 1, j) != 0.0) acc4 = f4fma(cf.cf[S - 1][j], kj, acc4);
                    if (S == 7 && dp_e(j) != 0.0) e4 = f4fma(cf.e[j], kj, e4);
                }
            }
            V[k] = f4mask(acc4, nib);
            sm.sv[((size_t)vs * 3 + k) * nt + i] = V[k];
            if (S == 7 && inner) sm.es[((size_t)(g & 1) * 3 + k) * nt + i] = e4;
        }
        sm.pr[(size_t)vs * nt + i] = (unsigned char)nib;
    };
    QuadRaw rw;
    // plane 0 was issued by stage_begin
    rw.idx = pp.fidx;
    rw.nib = (unsigned)pp.fnib;
    rw.inner = pp.finner != 0;
    float4 Vm[3], V0[3], Vp[3];
    unsigned nm = 0, n0 = 0, np_ = 0;
    int i0 = -1, ip = -1;
    bool in0 = false, inp = false;
    cp_async_wait<0>();
    combine(0, rw, V0, n0, i0, in0);
    quad_issue<S, HU>(c, sm, mn, 1, gend, pp.ci, r, qx, corner, inner_pos, rw);
    cp_async_commit();
#pragma unroll
    for (int k = 0; k < 3; k++) Vm[k] = V0[k];
    nm = n0;
    cp_async_wait<0>();
    combine(1, rw, V0, n0, i0, in0);
    quad_issue<S, HU>(c, sm, mn, 2, gend, pp.ci, r, qx, corner, inner_pos, rw);
    cp_async_commit();
    for (int p = 1; p <= gend - 2; p++) {
        load_rows(p + AHEAD);
        cp_async_wait<0>();   // this thread's copies of plane p+1
        combine(p + 1, rw, Vp, np_, ip, inp);
        quad_issue<S, HU>(c, sm, mn, p + 2, gend, pp.ci, r, qx, corner, inner_pos, rw);
        cp_async_commit();
        __syncthreads();
        if (in0)
            quad_cell<S, HU>(c, sm, kout, mnew, cf, p, Vm, V0, Vp, nm, n0, np_, i0, tslot, rslot,
                             acc);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            Vm[k] = V0[k];
            V0[k] = Vp[k];
        }
        nm = n0;
        n0 = np_;
        i0 = ip;
        in0 = inp;
    }
    cp_async_wait<0>();
}

}  // namespace cmx
