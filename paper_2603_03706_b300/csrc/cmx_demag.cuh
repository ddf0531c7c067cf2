// Full magnetostatic demag field of a stage value (sm_103a), evaluated by the team of blocks
// before the stage's cell pass when Ctx::fd is set.
//
// B_d = -mu0 Ms N * m_tot (a convolution over the magnetic cells with the cell-pair tensor, see
// cmx_demag_api.cu) by zero-padded FFTs of size Lx x Ly x Lz.  Only the first nx, ny, nz
// entries of each axis are nonzero on input and needed on output, so the five passes below
// transform only the lines that carry data; each pass hands its lines to the blocks of the
// team, transforms them in shared memory (radix-2, bit-reversed input) and ends with a team
// barrier:
//   1. x lines (y < ny, z < nz) of the three components of the stage's total moment
//   2. y lines (all kx, z < nz)
//   3. z lines (all kx, ky): forward, H = K^ M with the real tensor spectrum (which carries the
//      factor -mu0 Ms / (Lx Ly Lz)), inverse, z < nz kept
//   4. inverse y lines (all kx, z < nz), y < ny kept
//   5. inverse x lines (y < ny, z < nz): the real part at the magnetic cells -> Ctx::bd
// The work array holds nz planes of Ly x Lx complex values per component.  Everything that
// another block wrote (stage values, the work array) is read through L2 (ld.global.cg).
#pragma once

#include "cmx_stage.cuh"

namespace cmx {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int bit_reverse(int n, int lg)
{
    return lg == 0 ? 0 : (int)(__brev((unsigned)n) >> (32 - lg));
}

// In-place radix-2 transforms of nl lines of length L = 2^lg in shared memory (line l at
// s + l * L), input in bit-reversed order, output in natural order; tw[k] = e^{-2 pi i k / L},
// k < L/2; inv: conjugate twiddles (unscaled inverse).  Ends with a block barrier.
static __device__ void smem_fft(float2 *s, int L, int lg, int nl, const float2 *tw, bool inv)
{
    const int half = L >> 1, nb = nl * half;
    for (int h = 1; h < L; h <<= 1) {
        const int tstep = half / h;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int line = b / half, j = b - line * half;
            const int k = j & (h - 1), i0 = line * L + ((j - k) << 1) + k, i1 = i0 + h;
            float2 w = __ldg(tw + k * tstep);
            if (inv) w.y = -w.y;
            const float2 a = s[i0], t = cmulf(s[i1], w);
            s[i0] = make_float2(a.x + t.x, a.y + t.y);
            s[i1] = make_float2(a.x - t.x, a.y - t.y);
        }
        __syncthreads();
    }
}

// Component k of the total moment sum_s m_S of stage S at compact index idx: m_n (S = 1),
// m_n + h a_21 k_1 (S = 2, formed exactly as the tile formation of stage 2 does) or the stored
// stage value (S >= 3).
template <int S, int NS>
__device__ __forceinline__ float stage_total(const Ctx &c, const float *mn, const float *k1,
                                             float c21, int idx, int k)
{
    float v = 0.f;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const size_t o = (size_t)(s * 3 + k) * c.ncell + idx;
        float m;
        if (S == 1) m = __ldcg(mn + o);
        else if (S == 2) m = fmaf(c21, __ldcg(k1 + o), __ldcg(mn + o));
        else m = __ldcg(c.msv[S & 1] + o);
        v = (s == 0) ? m : v + m;
    }
    return v;
}

// The five passes (see the file comment).  Returns false if a team barrier failed.
template <int S, class SM>
__device__ bool demag_field(const Ctx &c, const Team &tm, SM &sm, Local &L, const Coef &cf,
                            const float *mn)
{
    constexpr int NS = SM::NQ / 3;
    const int NT = blockDim.x;
    const int nx = c.nx, ny = c.ny, nz = c.nz, Lx = c.Lx, Ly = c.Ly, Lz = c.Lz;
    const size_t plane = (size_t)Ly * Lx, comp = (size_t)nz * plane;
    const size_t NK = (size_t)Lz * plane;
    float2 *A = c.dwork;
    const float *k1 = sm.kp[0];
    const float c21 = cf.cf[1][0];
    // two line buffers of max(2 NT, 3 L) complex values each, in the operand pool
    const int cap = max(2 * NT, 3 * max(Lx, max(Ly, Lz)));
    float2 *b0 = reinterpret_cast<float2 *>(sm.pool), *b1 = b0 + cap;
    __syncthreads();   // the pool may still be read by the previous stage

    // 1. x lines of the total moment
    {
        const int Ln = Lx, lg = c.lgx, U = max(1, cap / (3 * Ln)), nu = ny * nz;
        for (int u0 = tm.rank * U; u0 < nu; u0 += tm.nblk * U) {
            const int nl = min(U, nu - u0);
            for (int e = threadIdx.x; e < nl * 3 * Ln; e += NT) {
                const int x = e % Ln, line = e / Ln, j = line / 3, k = line - 3 * j;
                const int u = u0 + j, y = u % ny, z = u / ny;
                float v = 0.f;
                if (x < nx) {
                    const int idx = row_index(c, row_entry(c, y, z), x);
                    if (idx >= 0) v = stage_total<S, NS>(c, mn, k1, c21, idx, k);
                }
                b0[line * Ln + bit_reverse(x, lg)] = make_float2(v, 0.f);
            }
            __syncthreads();
            smem_fft(b0, Ln, lg, nl * 3, c.dtw[0], false);
            for (int e = threadIdx.x; e < nl * 3 * Ln; e += NT) {
                const int x = e % Ln, line = e / Ln, j = line / 3, k = line - 3 * j;
                const int u = u0 + j, y = u % ny, z = u / ny;
                A[k * comp + z * plane + (size_t)y * Lx + x] = b0[line * Ln + x];
            }
            __syncthreads();
        }
    }
    if (!grid_barrier<SM>(c, tm, L, 21)) return false;

    // 2. y lines (kx, z); consecutive threads take consecutive kx
    {
        const int Ln = Ly, lg = c.lgy, U = max(1, cap / (3 * Ln)), nu = Lx * nz;
        for (int u0 = tm.rank * U; u0 < nu; u0 += tm.nblk * U) {
            const int nl = min(U, nu - u0);
            for (int e = threadIdx.x; e < nl * 3 * Ln; e += NT) {
                const int y = e / (3 * nl), r = e - y * 3 * nl, k = r / nl, j = r - k * nl;
                const int u = u0 + j, kx = u % Lx, z = u / Lx;
                const float2 v = y < ny ? __ldcg(A + k * comp + z * plane + (size_t)y * Lx + kx)
                                        : make_float2(0.f, 0.f);
                b0[(j * 3 + k) * Ln + bit_reverse(y, lg)] = v;
            }
            __syncthreads();
            smem_fft(b0, Ln, lg, nl * 3, c.dtw[1], false);
            for (int e = threadIdx.x; e < nl * 3 * Ln; e += NT) {
                const int y = e / (3 * nl), r = e - y * 3 * nl, k = r / nl, j = r - k * nl;
                const int u = u0 + j, kx = u % Lx, z = u / Lx;
                A[k * comp + z * plane + (size_t)y * Lx + kx] = b0[(j * 3 + k) * Ln + y];
            }
            __syncthreads();
        }
    }
    if (!grid_barrier<SM>(c, tm, L, 22)) return false;

    // 3. z lines (kx, ky): forward, tensor product, inverse
    {
        const int Ln = Lz, lg = c.lgz, U = max(1, cap / (3 * Ln)), nu = Lx * Ly;
        for (int u0 = tm.rank * U; u0 < nu; u0 += tm.nblk * U) {
            const int nl = min(U, nu - u0);
            for (int e = threadIdx.x; e < nl * 3 * Ln; e += NT) {
                const int z = e / (3 * nl), r = e - z * 3 * nl, k = r / nl, j = r - k * nl;
                const int u = u0 + j;
                const float2 v = z < nz ? __ldcg(A + k * comp + z * plane + u)
                                        : make_float2(0.f, 0.f);
                b0[(j * 3 + k) * Ln + bit_reverse(z, lg)] = v;
            }
            __syncthreads();
            smem_fft(b0, Ln, lg, nl * 3, c.dtw[2], false);
            for (int e = threadIdx.x; e < nl * Ln; e += NT) {
                const int kz = e % Ln, j = e / Ln;
                const size_t ki = (size_t)kz * plane + (u0 + j);
                const float xx = __ldg(c.dk + ki), yy = __ldg(c.dk + NK + ki),
                            zz = __ldg(c.dk + 2 * NK + ki), xy = __ldg(c.dk + 3 * NK + ki),
                            xz = __ldg(c.dk + 4 * NK + ki), yz = __ldg(c.dk + 5 * NK + ki);
                const float2 mx = b0[(j * 3 + 0) * Ln + kz], my = b0[(j * 3 + 1) * Ln + kz],
                             mz = b0[(j * 3 + 2) * Ln + kz];
                const int r = bit_reverse(kz, lg);
                b1[(j * 3 + 0) * Ln + r] = make_float2(xx * mx.x + xy * my.x + xz * mz.x,
                                                       xx * mx.y + xy * my.y + xz * mz.y);
                b1[(j * 3 + 1) * Ln + r] = make_float2(xy * mx.x + yy * my.x + yz * mz.x,
                                                       xy * mx.y + yy * my.y + yz * mz.y);
                b1[(j * 3 + 2) * Ln + r] = make_float2(xz * mx.x + yz * my.x + zz * mz.x,
                                                       xz * mx.y + yz * my.y + zz * mz.y);
            }
            __syncthreads();
            smem_fft(b1, Ln, lg, nl * 3, c.dtw[2], true);
            for (int e = threadIdx.x; e < nl * 3 * nz; e += NT) {
                const int z = e / (3 * nl), r = e - z * 3 * nl, k = r / nl, j = r - k * nl;
                A[k * comp + z * plane + (u0 + j)] = b1[(j * 3 + k) * Ln + z];
            }
            __syncthreads();
        }
    }
    if (!grid_barrier<SM>(c, tm, L, 23)) return false;

    // 4. inverse y lines (kx, z), y < ny kept
    {
        const int Ln = Ly, lg = c.lgy, U = max(1, cap / (3 * Ln)), nu = Lx * nz;
        for (int u0 = tm.rank * U; u0 < nu; u0 += tm.nblk * U) {
            const int nl = min(U, nu - u0);
            for (int e = threadIdx.x; e < nl * 3 * Ln; e += NT) {
                const int y = e / (3 * nl), r = e - y * 3 * nl, k = r / nl, j = r - k * nl;
                const int u = u0 + j, kx = u % Lx, z = u / Lx;
                b0[(j * 3 + k) * Ln + bit_reverse(y, lg)] =
                    __ldcg(A + k * comp + z * plane + (size_t)y * Lx + kx);
            }
            __syncthreads();
            smem_fft(b0, Ln, lg, nl * 3, c.dtw[1], true);
            for (int e = threadIdx.x; e < nl * 3 * ny; e += NT) {
                const int y = e / (3 * nl), r = e - y * 3 * nl, k = r / nl, j = r - k * nl;
                const int u = u0 + j, kx = u % Lx, z = u / Lx;
                A[k * comp + z * plane + (size_t)y * Lx + kx] = b0[(j * 3 + k) * Ln + y];
            }
            __syncthreads();
        }
    }
    if (!grid_barrier<SM>(c, tm, L, 24)) return false;

    // 5. inverse x lines (y, z): the field at the magnetic cells
    {
        const int Ln = Lx, lg = c.lgx, U = max(1, cap / (3 * Ln)), nu = ny * nz;
        for (int u0 = tm.rank * U; u0 < nu; u0 += tm.nblk * U) {
            const int nl = min(U, nu - u0);
            for (int e = threadIdx.x; e < nl * 3 * Ln; e += NT) {
                const int x = e % Ln, line = e / Ln, j = line / 3, k = line - 3 * j;
                const int u = u0 + j, y = u % ny, z = u / ny;
                b0[line * Ln + bit_reverse(x, lg)] =
                    __ldcg(A + k * comp + z * plane + (size_t)y * Lx + x);
            }
            __syncthreads();
            smem_fft(b0, Ln, lg, nl * 3, c.dtw[0], true);
            for (int e = threadIdx.x; e < nl * 3 * nx; e += NT) {
                const int x = e % nx, line = e / nx, j = line / 3, k = line - 3 * j;
                const int u = u0 + j, y = u % ny, z = u / ny;
                const int idx = row_index(c, row_entry(c, y, z), x);
                if (idx >= 0) c.bd[(size_t)k * c.ncell + idx] = b0[line * Ln + x].x;
            }
            __syncthreads();
        }
    }
    return grid_barrier<SM>(c, tm, L, 25);
}

}  // namespace cmx
