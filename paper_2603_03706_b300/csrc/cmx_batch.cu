// Batched integrator: one persistent cooperative launch advances many independent problems
// (kernel in cmx_batch_kernel.cuh, instantiated per tile shape in cmx_batch_t*.cu); the
// per-launch bookkeeping kernels, the drive and the spectral map.
#include "cmx_engine.cuh"
#include "cmx_kernels.h"

namespace cmx {

// Stream-ordered start of a batch launch: reset every instance's per-launch counters.
__global__ void batch_prep_kernel(Ctl *const *ctls, int n, long long max_attempts)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Ctl *c = ctls[i];
        c->done = 0;
        c->launch_attempts = 0;
        c->max_launch_attempts = max_attempts;
        c->bar_count = 0;
        c->skip_block = -1;
    }
}

// Number of instances that still have to run (t < T and no error) into *pending.
__global__ void batch_pending_kernel(Ctl *const *ctls, int n, int *pending)
{
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Ctl *c = ctls[i];
        mine += (c->status == 0 && c->t < c->T) ? 1 : 0;
    }
    atomicAdd(&s, mine);
    __syncthreads();
    if (threadIdx.x == 0) *pending = s;
}

template <int NS, int WX, int WY>
cudaError_t batch_launch_tiles(const BatchArgs &b, int blocks, cudaStream_t s);
template <int NS, int WX, int WY>
int batch_occupancy_tiles();

#define CMX_BATCH_VARIANTS(X) X(1, 32, 4) X(1, 32, 8) X(1, 32, 16) X(2, 32, 4) X(2, 32, 8)

cudaError_t launch_batch(const BatchArgs &b, int nsub, int bx, int by, int blocks, cudaStream_t s)
{
#define X(n, a, c) if (nsub == n && bx == a && by == c) return batch_launch_tiles<n, a, c>(b, blocks, s);
    CMX_BATCH_VARIANTS(X)
#undef X
    return cudaErrorInvalidValue;
}

int batch_blocks_per_sm(int nsub, int bx, int by)
{
#define X(n, a, c) if (nsub == n && bx == a && by == c) return batch_occupancy_tiles<n, a, c>();
    CMX_BATCH_VARIANTS(X)
#undef X
    return 0;
}

__global__ void batch_drive_kernel(Ctx *ctx, int n, DriveArgs d)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Ctx &c = ctx[i];
        for (int q = 0; q < MAXN; q++) {
            c.drive_re[q] = q < c.nmodes ? d.re[q] : 0.0;
            c.drive_im[q] = q < c.nmodes ? d.im[q] : 0.0;
        }
        c.drive_t0 = d.t0;
        c.drive_inv_sigma = d.inv_sigma;
        c.has_drive = d.on && c.nmodes > 0;
    }
}

cudaError_t launch_batch_drive(Ctx *ctx, int n, const DriveArgs &d, cudaStream_t s)
{
    batch_drive_kernel<<<(n + 127) / 128, 128, 0, s>>>(ctx, n, d);
    return cudaGetLastError();
}

// Spectral map: P_i(f) = | sum_k w_k a_{i,mode}(t_k) e^{+2 pi i f t_k} |^2 over the uniform trace
// samples with t_k >= t_start, w = Hann window over those samples (the e^{-i w t} convention of
// the cavity amplitude puts a mode at +f).  Block (instance, chunk of 128 frequencies), one
// thread per frequency; the samples pass through shared memory; the phasor advances by the
// constant sample step in FP64 and is recomputed exactly every 64 samples.
__global__ void batch_spectrum_kernel(const SpecInst *si, double f0, double df, int nf,
                                      double t_start, double *out)
{
    __shared__ double st[256], sr[256], sim_[256];
    const SpecInst I = si[blockIdx.x];
    const int fi = blockIdx.y * blockDim.x + threadIdx.x;
    const double f = f0 + df * fi;
    int n = (int)min((long long)I.cap, *(const volatile long long *)&I.ctl->trace_n);
    int k0 = 0;
    while (k0 < n && I.t[k0] < t_start) k0++;
    const int K = n - k0;
    double accr = 0.0, acci = 0.0;
    if (I.re >= 0 && K >= 2) {
        const double dt = I.t[k0 + 1] - I.t[k0];
        double sp, cp, sd, cd;
        sincospi(2.0 * f * dt - 2.0 * floor(f * dt), &sd, &cd);   // step phasor e^{2 pi i f dt}
        double pr = 1.0, pi = 0.0;
        for (int base = 0; base < K; base += 256) {
            const int m = min(256, K - base);
            __syncthreads();
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                const int k = k0 + base + j;
                const double w = 0.5 - 0.5 * cospi(2.0 * (double)(base + j) / (double)(K - 1));
                st[j] = I.t[k];
                sr[j] = w * I.a[(size_t)k * I.q + I.re];
                sim_[j] = w * I.a[(size_t)k * I.q + I.re + 1];
            }
            __syncthreads();
            if (fi < nf)
                for (int j = 0; j < m; j++) {
                    if ((j & 63) == 0) {   // exact phasor at this sample
                        const double x = f * st[j];
                        sincospi(2.0 * (x - floor(x)), &sp, &cp);
                        pr = cp;
                        pi = sp;
                    }
                    accr += sr[j] * pr - sim_[j] * pi;
                    acci += sr[j] * pi + sim_[j] * pr;
                    const double nr = pr * cd - pi * sd;
                    pi = pr * sd + pi * cd;
                    pr = nr;
                }
        }
    }
    if (fi < nf) out[(size_t)blockIdx.x * nf + fi] = accr * accr + acci * acci;
}

cudaError_t launch_batch_spectrum(const SpecInst *si, int n, double f0, double df, int nf,
                                  double t_start, double *out, cudaStream_t s)
{
    dim3 grid(n, (nf + 127) / 128);
    batch_spectrum_kernel<<<grid, 128, 0, s>>>(si, f0, df, nf, t_start, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_prep(Ctl *const *ctls, int n, long long max_attempts, cudaStream_t s)
{
    batch_prep_kernel<<<(n + 255) / 256, 256, 0, s>>>(ctls, n, max_attempts);
    return cudaGetLastError();
}

cudaError_t launch_batch_pending(Ctl *const *ctls, int n, int *pending, cudaStream_t s)
{
    batch_pending_kernel<<<1, 256, 0, s>>>(ctls, n, pending);
    return cudaGetLastError();
}

}  // namespace cmx
