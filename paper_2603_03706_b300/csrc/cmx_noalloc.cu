// Right-hand-side evaluation that allocates no device memory (cmx_eval_rhs_noalloc).
//
// Some callers cannot call cudaMalloc: plug-ins inside a host program whose own allocator owns
// all device memory, or services under a fixed device-memory budget that must not meet an
// out-of-memory error after start-up.  This entry point evaluates f(m, a) with the same stage kernel
// as cmx_eval_rhs but takes every scratch buffer (compact layout tables, compact m and slope,
// control block) from one file-scope device array of CMX_NOALLOC_SCRATCH_BYTES.
// That array exists on every device that loads the library, from load until process exit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cmx_kernels.h"
#include "cmx_layout.h"

using namespace cmx;

namespace {

constexpr size_t SCRATCH_BYTES = CMX_NOALLOC_SCRATCH_BYTES;
constexpr int MAX_DEVICES = 64;

// The shared scratch.  Host code must not use this name as a device address: on the host it
// is a stand-in symbol; the device address comes from cudaGetSymbolAddress (see scratch_base).
__device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

void *g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_base(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

__global__ void na_gather(const float *dense, float *compact, const int *box_of_cell,
                          const uint32_t *active, int ncell, long long nbox, int nq)
{
    const long long total = (long long)nq * ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / ncell), c = (int)(i - (long long)q * ncell);
        const bool on = !active || ((active[c >> 5] >> (c & 31)) & 1u);
        compact[i] = on ? dense[q * nbox + box_of_cell[c]] : 0.f;
    }
}

__global__ void na_scatter(const float *compact, float *dense, const int *box_of_cell,
                           const uint32_t *active, int ncell, long long nbox, int nq)
{
    const long long total = (long long)nq * ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / ncell), c = (int)(i - (long long)q * ncell);
        const bool on = !active || ((active[c >> 5] >> (c & 31)) & 1u);
        if (on) dense[q * nbox + box_of_cell[c]] = compact[i];
    }
}

// Bump allocator over the scratch (256-byte aligned pieces).
struct Carve {
    unsigned char *base;
    size_t used = 0;
    template <class T>
    T *take(size_t n)
    {
        const size_t bytes = (std::max<size_t>(n, 1) * sizeof(T) + 255) & ~(size_t)255;
        if (used + bytes > SCRATCH_BYTES) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

int grid_blocks(long long n) { return (int)std::min<long long>(1024, (n + 255) / 256); }

}  // namespace

extern "C" int cmx_eval_rhs_noalloc(const cmx_grid *grid, const uint8_t *mask,
                                    const cmx_material *mat, const cmx_modes *modes,
                                    const float *m, const double *a, float *dm, double *da,
                                    double *mm, void *stream)
{
    if (!grid || !mask || !mat || !m || !dm) return CMX_EINVAL;
    const int N = modes ? modes->n_modes : 0;
    if (grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0 || grid->nx > 65535 ||
        (grid->nsub != 1 && grid->nsub != 2) || N < 0 || N > MAXN || !(mat->Ms > 0) ||
        !(mat->gamma > 0) || !(grid->cx > 0) || !(grid->cy > 0) || !(grid->cz > 0))
        return CMX_EINVAL;
    if (N > 0 && (!modes->omega || !modes->kappa || !modes->g_re || !modes->g_im)) return CMX_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    const long long nbox = (long long)grid->nx * grid->ny * grid->nz;
    if (nbox > (1LL << 31) - 1) return CMX_EINVAL;   // box indices are 32-bit
    const int nq = 3 * grid->nsub;

    // host-side layout and partition (host memory only)
    Layout lay;
    build_layout(lay, grid->nx, grid->ny, grid->nz, mask);
    if (lay.ncell_mag == 0) return CMX_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CMX_ECUDA;
    const int bx = 32, by = 8;
    const bool has_u = N > 0 && modes->u;
    // bound on |u| for the fixed-point overlap sums: measured over the magnetic cells for host
    // profiles (as cmx_create does), 256 for device profiles (a larger value stops the
    // evaluation with CMX_ENAN through the range check of the block sums)
    double umax = 1.0;
    if (has_u && !modes->u_on_device) {
        for (int n = 0; n < N; n++)
            for (long long i = 0; i < nbox; i++)
                if (mask[i]) umax = std::max(umax, (double)std::fabs(modes->u[n * nbox + i]));
        if (!(umax < 1e30)) return CMX_EINVAL;   // non-finite profile
    } else if (has_u) {
        umax = 256.0;
    }
    const int occ = single_blocks_per_sm(grid->nsub, bx, by, has_u);
    if (occ <= 0) return CMX_ECUDA;
    const std::vector<Column> cols = build_columns(lay, bx, by);
    long long P = 0;
    for (const Column &c : cols) P += c.zhi - c.zlo;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)occ * nsm, (P + 3) / 4));
    std::vector<int4> segs;
    std::vector<int> begin;
    if (!build_segments(cols, blocks, segs, begin)) return CMX_EINVAL;   // too many tile columns

    // carve the scratch; reject problems that do not fit
    void *base = nullptr;
    if (scratch_base(&base) != cudaSuccess) return CMX_ECUDA;
    Carve cv{static_cast<unsigned char *>(base)};
    const size_t nc = (size_t)lay.ncell;
    int2 *rows = cv.take<int2>(lay.rows.size());
    int *box = cv.take<int>(nc);
    uint32_t *act = lay.padded ? cv.take<uint32_t>((nc + 31) / 32) : nullptr;
    int4 *tiles = cv.take<int4>(segs.size());
    int *sbeg = cv.take<int>(begin.size());
    float *uc = has_u ? cv.take<float>((size_t)N * nc) : nullptr;
    float *mc = cv.take<float>((size_t)nq * nc);
    float *kc = cv.take<float>((size_t)nq * nc);
    Ctl *ctl = cv.take<Ctl>(1);
    float *udense = has_u && !modes->u_on_device ? cv.take<float>((size_t)N * nbox) : nullptr;
    if (!rows || !box || (lay.padded && !act) || !tiles || !sbeg || (has_u && !uc) || !mc ||
        !kc || !ctl || (has_u && !modes->u_on_device && !udense))
        return CMX_ESCRATCH;   // larger than CMX_NOALLOC_SCRATCH_BYTES

    // tables and inputs into the scratch (every field the kernel reads is written here)
    const std::vector<uint32_t> bits = lay.padded ? active_bits(lay) : std::vector<uint32_t>();
    Ctl c0;
    memset(&c0, 0, sizeof c0);
    for (int q = 0; q < 2 * N; q++) c0.a[q] = a ? a[q] : 0.0;
    for (int j = 0; j < 7; j++) c0.kphys[j] = j;
    c0.dt = 1e-13;
    c0.T = 1.0;
    c0.skip_block = -1;
    c0.max_launch_attempts = 1;
    cudaError_t e = cudaSuccess;
    auto h2d = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    h2d(rows, lay.rows.data(), lay.rows.size() * sizeof(int2));
    h2d(box, lay.box_of_cell.data(), nc * sizeof(int));
    if (act) h2d(act, bits.data(), bits.size() * sizeof(uint32_t));
    h2d(tiles, segs.data(), segs.size() * sizeof(int4));
    h2d(sbeg, begin.data(), begin.size() * sizeof(int));
    h2d(ctl, &c0, sizeof c0);
    if (e != cudaSuccess) return CMX_ECUDA;
    if (has_u) {
        const float *usrc = modes->u;
        if (!modes->u_on_device) {
            h2d(udense, modes->u, (size_t)N * nbox * sizeof(float));
            usrc = udense;
        }
        na_gather<<<grid_blocks((long long)N * nc), 256, 0, s>>>(usrc, uc, box, act, (int)nc, nbox, N);
    }
    na_gather<<<grid_blocks((long long)nq * nc), 256, 0, s>>>(m, mc, box, act, (int)nc, nbox, nq);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return CMX_ECUDA;

    // the stage kernel, stage 1 only
    Ctx c;
    memset(&c, 0, sizeof c);
    c.nx = grid->nx;
    c.ny = grid->ny;
    c.nz = grid->nz;
    c.nsub = grid->nsub;
    c.nmodes = N;
    c.ncell = (int)nc;
    c.ncell_mag = lay.ncell_mag;
    c.rows = rows;
    c.active = lay.holes ? act : nullptr;   // the row spans exclude the padding
    c.tiles = tiles;
    c.seg_begin = sbeg;
    c.ntiles = (int)segs.size();
    c.bz = 4;
    c.u = uc;
    c.m[0] = c.m[1] = mc;
    for (int j = 0; j < 7; j++) c.k[j] = kc;
    const double exch = 2.0 * mat->Aex / mat->Ms;
    c.wx = (float)(exch / (grid->cx * grid->cx));
    c.wy = (float)(exch / (grid->cy * grid->cy));
    c.wz = (float)(exch / (grid->cz * grid->cz));
    c.anis = (float)(2.0 * mat->Ku / mat->Ms);
    const double mu0 = 4.0e-7 * M_PI;
    for (int k = 0; k < 3; k++) {
        c.ku[k] = (float)mat->ku_axis[k];
        c.B0[k] = (float)mat->B0[k];
        c.dmg[k] = (float)(mu0 * mat->Ms * mat->Ndemag[k]);
    }
    c.BE = grid->nsub == 2 ? (float)mat->BE : 0.f;
    c.pre = (float)(-mat->gamma / (1.0 + mat->alpha * mat->alpha));
    c.alpha = (float)mat->alpha;
    for (int n = 0; n < N; n++) {
        c.omega[n] = modes->omega[n];
        c.kappa[n] = modes->kappa[n];
        c.gre[n] = modes->g_re[n];
        c.gim[n] = modes->g_im[n];
        c.gbre[n] = modes->g_re[n];   // reciprocal coupling
        c.gbim[n] = modes->g_im[n];
    }
    c.two_over_gamma = 2.0 / mat->gamma;
    c.inv_nmag = 1.0 / (double)lay.ncell_mag;
    c.red_scale = overlap_scale(umax * (double)lay.ncell_mag);
    c.umax = (float)umax;
    c.rtol = 1e-6;
    c.a_ref = 1e-3;
    c.dt_min = 1e-18;
    c.dt_max = 1e-11;
    c.ctl = ctl;
    c.timeout_ns = 2000000000LL;
    c.stage_only = 1;
    if (launch_single(c, bx, by, blocks, s) != cudaSuccess) return CMX_ECUDA;

    // outputs: dm (device, dense box, zero outside the mask), da and mm (host)
    if (cudaMemsetAsync(dm, 0, (size_t)nq * nbox * sizeof(float), s) != cudaSuccess) return CMX_ECUDA;
    na_scatter<<<grid_blocks((long long)nq * nc), 256, 0, s>>>(kc, dm, box, act, (int)nc, nbox, nq);
    Ctl hc;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CMX_ECUDA;
    if (hc.status) return hc.status;
    for (int q = 0; q < 2 * N; q++) {
        if (da) da[q] = hc.ka[0][q];
        if (mm) mm[q] = hc.mm_n[q];
    }
    return CMX_OK;
}
