// Single-block integrator for small grids (sm_103a).
//
// A grid of a few hundred to about a thousand magnetic cells (the 280-cell 8^3 sphere of the
// single-mode Rabi and anticrossing runs of Sec. IV A-B) is integrated by ONE block of 256
// threads that keeps, for every magnetic cell, m_n and the new state, the stage value, the seven
// slopes, the error partial, the mode profiles and a neighbour table in shared memory.  A stage is
// one block-wide pass over the cells (field, slope and the cell's next stage value; stage 2 also
// a pass forming its stage values), the overlap sums are
// block sums in shared memory with the same fixed-point digits as the multi-block reduction, and
// the cavity update and the step-size controller are the engine's own (warp 0).  No stage touches
// global memory except for the step log and the trace, and a stage costs two or three block
// barriers instead of a grid barrier through L2.  The per-cell arithmetic is the tiled kernel's
// (cell_slope, the same combine order), so the two integrate the same discrete system.
#include "cmx_engine.cuh"
#include "cmx_kernels.h"

namespace cmx {

constexpr int SMALL_NT = 256;
constexpr int SMALL_NW = SMALL_NT / 32;

size_t small_smem_bytes(int nm, int nsub, int nmodes, bool has_u)
{
    const size_t nq = 3 * (size_t)nsub;
    return ((2 + 2 + 1 + 7) * nq + (has_u ? (size_t)nmodes : 0)) * nm * sizeof(float) +
           6 * (size_t)nm * sizeof(int);
}

// Block-level scratch of the overlap sums (fixed-point digits per warp, then per component in
// units of 1 / red_scale) and of the error maximum.
struct SmallRed {
    int dig[SMALL_NW][2 * MAXN][2];
    unsigned wmax[SMALL_NW];
    long long sum[2 * MAXN];
    unsigned emax;
    int bad;
};

// Block sums of the per-thread overlap accumulators and block max of |e_m|: each thread's FP32
// partial is scaled by L.tscale and split into two int32 digits (integer part and remainder in
// units of 2^-20), summed exactly over the warp (redux) and the block (int64), and converted to
// the grid units 1 / red_scale, exactly as the multi-block reduction forms one block's share.
__device__ void small_block_sums(const Ctx &c, const Local &L, const Acc &acc, SmallRed &R)
{
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
            const float vh = rintf(v);
            const int dh = __reduce_add_sync(0xffffffffu, __float2int_rn(vh));
            const int dl = __reduce_add_sync(0xffffffffu, __float2int_rn((v - vh) * 1048576.f));
            if (lane == 0) {
                R.dig[warp][2 * n + k][0] = dh;
                R.dig[warp][2 * n + k][1] = dl;
            }
        }
    }
    const unsigned e = __reduce_max_sync(0xffffffffu, __float_as_uint(acc.emax));
    if (lane == 0) R.wmax[warp] = e;
    if (bad) atomicOr(&R.bad, 1);
    __syncthreads();
    if (threadIdx.x < 2 * c.nmodes) {
        long long sh = 0, sl = 0;
        for (int w = 0; w < SMALL_NW; w++) {
            sh += R.dig[w][threadIdx.x][0];
            sl += R.dig[w][threadIdx.x][1];
        }
        long long v = sh * (1ll << 20) + sl;
        const int d = L.tshift;
        R.sum[threadIdx.x] = d >= 0 ? v * (1ll << d) : (v + (1ll << (-d - 1))) >> (-d);
    }
    if (threadIdx.x == SMALL_NT - 1) {
        unsigned m = 0u;
        for (int w = 0; w < SMALL_NW; w++) m = max(m, R.wmax[w]);
        R.emax = m;
    }
    __syncthreads();
}

struct SmallBuf {
    float *mb0, *mb1;      // the two state buffers (index = the control block's mcur)
    float *ms[2];          // stage values: stage S reads ms[S & 1], writes m_{S+1} to the other
    float *es, *kk;        // error partial, slopes [physical][q][cell]
    const float *uu;       // profiles [n][cell]
    const int *nb;         // neighbours [-x, +x, -y, +y, -z, +z][cell], -1 = none
};

// One Dormand-Prince stage of all cells (see the file comment); the controller follows.
template <int NS, bool HU, int S>
__device__ void small_stage(const Ctx &c, int nm, const SmallBuf &b, Local &L, Coef &cf,
                            SmallRed &R)
{
    constexpr int NQ = 3 * NS;
    const int tid = threadIdx.x;
    const size_t V = (size_t)NQ * nm;
    const float *mn = L.mcur ? b.mb1 : b.mb0;
    float *mnew = L.mcur ? b.mb0 : b.mb1;
    if (S <= 2) {
        if (tid < 32) cavity_stage_value<S>(L, cf, tid, tid < 2 * c.nmodes);
        if (S == 2 && tid >= 32 && tid < 32 + 36) attempt_coefficients(cf, L, L.h, tid - 32);
        if (S == 2 && tid == 96) cf.h = (float)L.h;
        __syncthreads();
    }
    // stage values: stage 2 forms m_2 = m_n + h a_21 k_1 in a pass of its own (the step size is
    // known only when the attempt starts); stages 2..6 form the next stage value
    // m_{S+1} = m_n + sum_{j<=S} (h a_{S+1,j}) k_j of their cell right after its slope (and stage
    // 6 the error partial sum_{j<=6} E_j k_j), in the tiled kernel's order of operations, so
    // stages 3..7 need no pass and no barrier before their field pass
    const float *src = S == 1 ? mn : b.ms[S & 1];
    if (S == 2) {
        for (int i = tid; i < nm; i += SMALL_NT)
#pragma unroll
            for (int q = 0; q < NQ; q++)
                b.ms[0][q * nm + i] =
                    fmaf(cf.cf[1][0], b.kk[L.kphys[0] * V + q * nm + i], mn[q * nm + i]);
        __syncthreads();
    }
    Acc acc;
#pragma unroll
    for (int n = 0; n < MAXN; n++) acc.re[n] = acc.im[n] = 0.f;
    acc.emax = 0.f;
    float *kout = b.kk + L.kphys[S - 1] * V;
    for (int i = tid; i < nm; i += SMALL_NT) {
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
        cell_slope<NS, HU>(c, cf, m, B, ucell, bdem, acc, kv);
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
                        if (dp_a(S, j) != 0.0) a = fmaf(cf.cf[S][j], kj, a);
                        if (S == 6 && dp_e(j) != 0.0) e = fmaf(cf.e[j], kj, e);
                    }
                    b.ms[(S + 1) & 1][q * nm + i] = fmaf(cf.cf[S][S - 1], kv[s][k], a);
                    if (S == 6) b.es[q * nm + i] = fmaf(cf.e[5], kv[s][k], e);
                }
            }
            if (S == 7) {
                const float *mm = m[s];
                const float r = rsqrtf(mm[0] * mm[0] + mm[1] * mm[1] + mm[2] * mm[2]);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const int q = s * 3 + k;
                    mnew[q * nm + i] = mm[k] * r;
                    const float e7 = cf.h * fmaf(cf.e[6], kv[s][k], b.es[q * nm + i]);
                    acc.emax = nanmax(acc.emax, fabsf(e7));
                }
            }
        }
    }
    small_block_sums(c, L, acc, R);
    const long long sq = tid < 2 * c.nmodes ? R.sum[tid] : 0;
    float emax = 0.f;
    if (S == 7 && tid < 32) emax = R.bad ? __int_as_float(0x7fffffff) : __uint_as_float(R.emax);
    const Team tm{0, 1, nullptr};
    controller<S>(c, tm, L, cf, sq, emax);
    __syncthreads();
}

struct SmallArgs {
    Ctx c;
    const int *sidx;   // [nm] stored (compact) index of magnetic cell i
    const int *snb;    // [6][nm] neighbour table (see SmallBuf)
    int nm;
};

template <int NS, bool HU>
__global__ void __launch_bounds__(SMALL_NT, 1) small_kernel(SmallArgs A)
{
    extern __shared__ __align__(16) float sh[];
    __shared__ Local L;
    __shared__ Coef cf;
    __shared__ SmallRed R;
    __shared__ int s_stop;
    constexpr int NQ = 3 * NS;
    const Ctx &c = A.c;
    const int nm = A.nm, tid = threadIdx.x;
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
        // fixed-point scale of the per-thread overlap partials (ceil(nm / 256) cells each)
        const int P = (nm + SMALL_NT - 1) / SMALL_NT;
        const float bound = 2.f * (float)(P > 1 ? P : 1) * fmaxf(c.umax, 1.f);
        const int k = 24 - (int)ceilf(log2f(bound));
        L.tscale = ldexpf(1.f, k);
        L.tshift = ilogb(c.red_scale) - k - 20;
        R.bad = 0;
    }
    if (tid < 2 * c.nmodes) component_constants(c, tid, L);
    if (tid >= 32 && tid < 39) cf.e[tid - 32] = (float)dp_e(tid - 32);
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
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            s_stop = L.status != 0 || L.done;
            if (!s_stop) attempt_size(c, L);
        }
        __syncthreads();
        if (s_stop) break;
        while (!L.k1_valid) small_stage<NS, HU, 1>(c, nm, b, L, cf, R);   // twice at a split boundary
        small_stage<NS, HU, 2>(c, nm, b, L, cf, R);
        small_stage<NS, HU, 3>(c, nm, b, L, cf, R);
        small_stage<NS, HU, 4>(c, nm, b, L, cf, R);
        small_stage<NS, HU, 5>(c, nm, b, L, cf, R);
        small_stage<NS, HU, 6>(c, nm, b, L, cf, R);
        small_stage<NS, HU, 7>(c, nm, b, L, cf, R);
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
                if (L.k1_valid) gk1[(size_t)q * c.ncell + si] = k1[q * nm + i];
            }
        }
    }
}

template <int NS, bool HU>
static cudaError_t small_launch_variant(const SmallArgs &a, cudaStream_t s)
{
    auto *fn = small_kernel<NS, HU>;
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
