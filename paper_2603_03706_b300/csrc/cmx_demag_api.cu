// Full magnetostatic demag: host set-up of the convolution kernel (cmx_set_demag).
//
// The demag field of the magnetic cells is the convolution B_d(r_i) = -mu0 Ms sum_j
// N(r_i - r_j) m_j with the cell-pair tensor of Newell, Williams & Dunlop (J. Geophys. Res. 98,
// 9551 (1993)): the field of a uniformly magnetised cuboid cell averaged over another.  Written
// with the negative second difference D_h q(X) = 2 q(X) - q(X - h) - q(X + h),
//   N_xx = D_cx D_cy D_cz f / (4 pi cx cy cz),  N_xy = D_cx D_cy D_cz g / (4 pi cx cy cz)
// and the other components by permuting the axes, f and g being Newell's closed forms.  The
// device evaluates the convolution with zero-padded FFTs of size Lx x Ly x Lz (powers of two,
// L >= 2n - 1); here the tensor is tabulated on the padded grid (negative displacements wrap
// around), transformed in FP64 on the host and stored, scaled by -mu0 Ms / (Lx Ly Lz), as six
// real FP32 spectra (each component is even or odd in every axis, so its spectrum is real).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "cmx_problem.h"

using namespace cmx;
using namespace cmx_host;

namespace {

using cd = std::complex<double>;

// Newell's f (even in x, y, z)
double nw_f(double x, double y, double z)
{
    x = std::fabs(x);
    y = std::fabs(y);
    z = std::fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z, r = std::sqrt(xx + yy + zz);
    double v = (2.0 * xx - yy - zz) * r / 6.0;
    if (y > 0 && xx + zz > 0) v += 0.5 * y * (zz - xx) * std::asinh(y / std::sqrt(xx + zz));
    if (z > 0 && xx + yy > 0) v += 0.5 * z * (yy - xx) * std::asinh(z / std::sqrt(xx + yy));
    if (x > 0 && y > 0 && z > 0) v -= x * y * z * std::atan(y * z / (x * r));
    return v;
}

// Newell's g (odd in x and y, even in z)
double nw_g(double x, double y, double z)
{
    const double s = ((x < 0) != (y < 0)) ? -1.0 : 1.0;
    x = std::fabs(x);
    y = std::fabs(y);
    z = std::fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z, r = std::sqrt(xx + yy + zz);
    double v = -x * y * r / 3.0;
    if (z > 0 && xx + yy > 0) v += x * y * z * std::asinh(z / std::sqrt(xx + yy));
    if (x > 0 && yy + zz > 0) v += y * (3.0 * zz - yy) / 6.0 * std::asinh(x / std::sqrt(yy + zz));
    if (y > 0 && xx + zz > 0) v += x * (3.0 * zz - xx) / 6.0 * std::asinh(y / std::sqrt(xx + zz));
    if (x > 0 && y > 0 && z > 0)
        v -= z * zz / 6.0 * std::atan(x * y / (z * r)) + 0.5 * z * yy * std::atan(x * z / (y * r)) +
             0.5 * z * xx * std::atan(y * z / (x * r));
    return s * v;
}

// D_hx D_hy D_hz q(X, Y, Z) / (4 pi hx hy hz), q = f (off = false) or g (off = true)
double nw_tensor(bool off, double X, double Y, double Z, double hx, double hy, double hz)
{
    const double w[3] = {-1.0, 2.0, -1.0};
    double acc = 0.0;
    for (int a = -1; a <= 1; a++)
        for (int b = -1; b <= 1; b++)
            for (int e = -1; e <= 1; e++) {
                const double x = X + a * hx, y = Y + b * hy, z = Z + e * hz;
                acc += w[a + 1] * w[b + 1] * w[e + 1] * (off ? nw_g(x, y, z) : nw_f(x, y, z));
            }
    return acc / (4.0 * M_PI * hx * hy * hz);
}

// In-place radix-2 FFT (forward, e^{-2 pi i k n / L}) of n lines of length L with element stride
// `st` and line starts from `start(line)`.
void fft_axis(std::vector<cd> &a, int L, size_t st, const std::vector<size_t> &starts)
{
    if (L <= 1) return;
    int lg = 0;
    while ((1 << lg) < L) lg++;
    std::vector<cd> tw(L / 2), buf(L);
    for (int k = 0; k < L / 2; k++) tw[k] = std::polar(1.0, -2.0 * M_PI * k / L);
    for (size_t s0 : starts) {
        for (int n = 0; n < L; n++) {
            int r = 0;
            for (int b = 0; b < lg; b++) r |= ((n >> b) & 1) << (lg - 1 - b);
            buf[r] = a[s0 + (size_t)n * st];
        }
        for (int h = 1; h < L; h <<= 1)
            for (int g = 0; g < L; g += 2 * h)
                for (int k = 0; k < h; k++) {
                    const cd t = tw[(size_t)k * (L / (2 * h))] * buf[g + k + h];
                    buf[g + k + h] = buf[g + k] - t;
                    buf[g + k] += t;
                }
        for (int n = 0; n < L; n++) a[s0 + (size_t)n * st] = buf[n];
    }
}

int pow2_at_least(int n)
{
    int L = 1;
    while (L < n) L <<= 1;
    return L;
}

int log2i(int L)
{
    int l = 0;
    while ((1 << l) < L) l++;
    return l;
}

void demag_free(cmx_problem *h)
{
    void *p[] = {h->dm_k, h->dm_work, h->dm_bd, h->dm_tw};
    for (void *q : p)
        if (q) cudaFree(q);
    h->dm_k = nullptr;
    h->dm_work = nullptr;
    h->dm_bd = nullptr;
    h->dm_tw = nullptr;
}

}  // namespace

void cmx_host::demag_release(cmx_problem *h) { demag_free(h); }

extern "C" int cmx_set_demag(cmx_problem *h, int mode)
{
    if (!h || (mode != 0 && mode != 1)) return fail(h, CMX_EINVAL, "demag mode must be 0 or 1");
    Ctx &c = h->base;
    const double mu0 = 4.0e-7 * M_PI;
    if (mode == 0) {
        for (int k = 0; k < 3; k++) c.dmg[k] = (float)(mu0 * h->mat.Ms * h->mat.Ndemag[k]);
        const bool was_full = c.fd != 0;
        c.fd = 0;
        demag_free(h);
        h->use_small = h->small_ok && h->small_default;
        // back to the launch shape of the diagonal factors (the full demag used every resident
        // block for its FFT passes)
        return was_full ? retile(h, h->bx, h->by) : CMX_OK;
    }
    if (h->base.traj_m)
        return fail(h, CMX_EINVAL, "the adjoint covers the diagonal demag factors only");
    const int nx = h->grid.nx, ny = h->grid.ny, nz = h->grid.nz;
    const int Lx = pow2_at_least(2 * nx - 1), Ly = pow2_at_least(2 * ny - 1),
              Lz = pow2_at_least(2 * nz - 1);
    if (Lx > CMX_DEMAG_MAX_FFT || Ly > CMX_DEMAG_MAX_FFT || Lz > CMX_DEMAG_MAX_FFT)
        return fail(h, CMX_EINVAL, "full demag: grid %dx%dx%d exceeds %d cells per axis", nx, ny,
                    nz, CMX_DEMAG_MAX_FFT / 2);
    const size_t NK = (size_t)Lx * Ly * Lz;
    const double cx = h->grid.cx, cy = h->grid.cy, cz = h->grid.cz;
    const double scale = -mu0 * h->mat.Ms / (double)NK;
    std::vector<float> spec(6 * NK);
    std::vector<cd> a(NK);
    std::vector<size_t> sx, sy, sz;
    for (int z = 0; z < Lz; z++)
        for (int y = 0; y < Ly; y++) sx.push_back(((size_t)z * Ly + y) * Lx);
    for (int z = 0; z < Lz; z++)
        for (int x = 0; x < Lx; x++) sy.push_back((size_t)z * Ly * Lx + x);
    for (int y = 0; y < Ly; y++)
        for (int x = 0; x < Lx; x++) sz.push_back((size_t)y * Lx + x);
    double worst_imag = 0.0, largest = 0.0;
    for (int comp = 0; comp < 6; comp++) {
        std::fill(a.begin(), a.end(), cd(0.0, 0.0));
        for (int k = -(nz - 1); k < nz; k++)
            for (int j = -(ny - 1); j < ny; j++)
                for (int i = -(nx - 1); i < nx; i++) {
                    // evaluated at |displacement| with the component's parity applied, so
                    // that entries of opposite displacements are exactly equal or opposite
                    // and the spectrum is real up to the transform's rounding (the far entries
                    // carry the cancellation error of the second differences, which differs
                    // with the summation order)
                    const double X = std::abs(i) * cx, Y = std::abs(j) * cy, Z = std::abs(k) * cz;
                    const int si = (i > 0) - (i < 0), sj = (j > 0) - (j < 0), sk = (k > 0) - (k < 0);
                    double v = 0.0;
                    switch (comp) {
                    case 0: v = nw_tensor(false, X, Y, Z, cx, cy, cz); break;             // xx
                    case 1: v = nw_tensor(false, Y, X, Z, cy, cx, cz); break;             // yy
                    case 2: v = nw_tensor(false, Z, Y, X, cz, cy, cx); break;             // zz
                    case 3: v = si * sj * nw_tensor(true, X, Y, Z, cx, cy, cz); break;    // xy
                    case 4: v = si * sk * nw_tensor(true, X, Z, Y, cx, cz, cy); break;    // xz
                    default: v = sj * sk * nw_tensor(true, Y, Z, X, cy, cz, cx); break;   // yz
                    }
                    const size_t o = (((size_t)((k + Lz) % Lz)) * Ly + (size_t)((j + Ly) % Ly)) * Lx +
                                     (size_t)((i + Lx) % Lx);
                    a[o] = cd(v, 0.0);
                }
        fft_axis(a, Lx, 1, sx);
        fft_axis(a, Ly, Lx, sy);
        fft_axis(a, Lz, (size_t)Lx * Ly, sz);
        for (size_t o = 0; o < NK; o++) {
            worst_imag = std::max(worst_imag, std::fabs(a[o].imag()));
            largest = std::max(largest, std::fabs(a[o].real()));
            spec[comp * NK + o] = (float)(scale * a[o].real());
        }
    }
    if (!(worst_imag <= 1e-9 * std::max(largest, 1e-300)))
        return fail(h, CMX_ECUDA, "demag spectrum is not real (%g)", worst_imag);
    // twiddles e^{-2 pi i k / L}, k < L/2, of the three axes
    std::vector<float2> tw;
    for (int L : {Lx, Ly, Lz})
        for (int k = 0; k < std::max(1, L / 2); k++)
            tw.push_back(make_float2((float)std::cos(2.0 * M_PI * k / L),
                                     (float)-std::sin(2.0 * M_PI * k / L)));
    demag_free(h);
    const int nq = 3 * h->grid.nsub;
    (void)nq;
    if (dalloc(&h->dm_k, 6 * NK) != cudaSuccess ||
        dalloc(&h->dm_work, (size_t)3 * nz * Ly * Lx) != cudaSuccess ||
        dalloc(&h->dm_bd, (size_t)3 * h->ncell) != cudaSuccess ||
        dalloc(&h->dm_tw, tw.size()) != cudaSuccess) {
        demag_free(h);
        return fail(h, CMX_ENOMEM, "full demag buffers");
    }
    CU(cudaMemcpy(h->dm_k, spec.data(), spec.size() * sizeof(float), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->dm_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CU(cudaMemset(h->dm_bd, 0, (size_t)3 * h->ncell * sizeof(float)));
    c.fd = 1;
    for (int k = 0; k < 3; k++) c.dmg[k] = 0.f;
    c.dk = h->dm_k;
    c.dwork = h->dm_work;
    c.bd = h->dm_bd;
    c.dtw[0] = h->dm_tw;
    c.dtw[1] = h->dm_tw + std::max(1, Lx / 2);
    c.dtw[2] = h->dm_tw + std::max(1, Lx / 2) + std::max(1, Ly / 2);
    c.Lx = Lx;
    c.Ly = Ly;
    c.Lz = Lz;
    c.lgx = log2i(Lx);
    c.lgy = log2i(Ly);
    c.lgz = log2i(Lz);
    h->use_small = false;   // the single-block integrator has no demag passes
    return retile(h, 32, 8);   // the kernels with the demag passes use 32 x 8 tiles
}
