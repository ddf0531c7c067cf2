/*
 * FP64 CPU oracle for the coupled LLG + N-cavity-mode system, integrated with an adaptive
 * Dormand-Prince 5(4) scheme.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header or constant table with the CUDA
 * path: everything below is written out again from the paper and from the published
 * Dormand-Prince tableau.
 *
 * What it computes (paper = "Multimode cavity magnonics in mumax+", arXiv 2603.03706):
 *   cavity ODEs      da_n/dt = (-i w_n - kappa_n) a_n + i g~_n <m^->_n          Eq. (12), (19)
 *   overlap          <m^->_n = (1/N_c) sum_{r in mask} u_n(r) (m_x - i m_y)(r)  Eq. (2), (18)
 *   feedback field   B_rf,x(r) = sum_n u_n(r) (2/gamma) Re[g~_n a_n]            Eq. (5), (13)
 *   magnetisation    LLG with Gilbert damping (Sec. II A), Landau-Lifshitz form:
 *                    dm/dt = -gamma/(1+alpha^2) [ m x B + alpha m x (m x B) ]
 *   effective field  B = exchange (6 neighbours, free surface) + uniaxial anisotropy + Zeeman
 *                    + diagonal demag + B_rf (+ inter-sublattice exchange -B_E m_other, AFM,
 *                    Sec. II G); for two sublattices the cavity couples to (m1 + m2)/2.
 *   time stepping    Dormand-Prince 5(4), FSAL; the paper only says "adaptive RK45" (Sec. III A).
 *   drive            optional eta_n(t) added to da_n/dt (Eq. (1), (12)), a Gaussian pulse
 *                    (Sec. IV A), evaluated at each stage's time t + c_s h.
 *   extensions       optional backward coupling gb~_n of the feedback field (nonreciprocal
 *                    coupling, Sec. II: h0 = 2 g_b / gamma) and self-Kerr -i K_n |a_n|^2 a_n.
 *   parametric pump  optional -i P_n exp(-i wp_n t) conj(a_n) added to da_n/dt at each stage's
 *                    time (Sec. V names parametric drives as a cavity-model swap without a
 *                    formula: this is the classical equation of the degenerate two-photon pump
 *                    H/hbar = (P e^{-i wp t} a^dag^2 + conj) / 2).
 *   adjoint          orc_rhs_vjp / orc_adjoint: reverse-mode derivative of the replayed steps
 *                    (not in the paper; the gradient form added beside the integrator).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - coupling sign +i g~ (Eq. (1)); complex g~ = g - i g_d feeds back through Re[g~ a]
 *   - the overlap is an average (1/N_c), Eq. (18)
 *   - exchange neighbours outside the mask or the box contribute nothing (free surface)
 *   - demag of a two-sublattice magnet acts on the total moment Ms (m1 + m2)
 *   - error norm: err = max( max|e_m| / rtol , max_n |e_a,n| / (rtol max(a_ref, |a|max)) ),
 *     accept iff err <= 1, dt *= clamp(0.9 err^(-1/5), 0.2, 5), no growth right after a reject
 *   - on accept m is renormalised per cell; the FSAL slope k7 is the slope at the
 *     un-normalised 5th-order point.
 *
 * Layout: dense box, x fastest, cell = x + nx*(y + ny*z).  m[(s*3 + c)*nbox + cell] for
 * sublattice s and component c.  Cavity amplitudes a[2n] = Re a_n, a[2n+1] = Im a_n.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENAN 4
#define ORC_ESTEPFAIL 5

static const double ORC_MU0 = 4.0e-7 * 3.14159265358979323846;

typedef struct {
    int nx, ny, nz, nsub, nmodes;
    double cx, cy, cz;
    const unsigned char *mask;
    double Ms, Aex, alpha, gamma, Ku, ku[3], B0[3], Nd[3], BE;
    const double *u; /* nmodes * nbox, or NULL: every profile is 1 */
    const double *omega, *kappa, *g_re, *g_im;
    /* external drive eta_n(t) = (drive_re + i drive_im)_n exp(-(t - drive_t0)^2 / (2 sigma^2))
       added to da_n/dt (Eq. (1), (12)); drive_re == NULL: no drive */
    const double *drive_re, *drive_im;
    double drive_t0, drive_sigma;
    /* nonreciprocal coupling: backward (cavity-to-magnon) coefficients of the feedback field,
       B_rf,x = sum_n u_n (2/gamma) Re[gb~_n a_n] (Sec. II, h0 = 2 g_b / gamma); NULL: gb~ = g~ */
    const double *gb_re, *gb_im;
    /* self-Kerr term -i K_n |a_n|^2 a_n of the cavity equation; NULL: none */
    const double *kerr;
    /* 1: the cavity amplitudes are held fixed (da/dt = 0, no drive): the magnet-only
       sub-integration of the operator-split scheme (orc_run_split) */
    int cavity_frozen;
    /* degenerate parametric pump -i P_n e^{-i wp_n t} conj(a_n) on da_n/dt, P_n = pump_re + i
       pump_im [rad/s], pump frequency pump_w [rad/s]; pump_re == NULL: none */
    const double *pump_re, *pump_im, *pump_w;
    /* full magnetostatic demag (NEXT-3 of the scope; Sec. II C-D, Eq. (9), (11)): the cell-pair
       demag tensor of every displacement (orc_demag_tensor); NULL: the diagonal factors Nd */
    const double *demag;
} orc_problem;

typedef struct {
    double rtol, a_ref, dt_min, dt_max;
} orc_solver;

/* Per-attempt record written by the drivers below. */
typedef struct {
    int cap, n;
    double *t;    /* time at the end of the attempt (accepted) or at its start (rejected) */
    double *dt;
    double *err;
    int *accepted;
    double *a;    /* cap * 2N: cavity amplitudes after the attempt (only for accepted) */
    double *mm;   /* cap * 2N: <m^->_n at the stage-7 point y_{n+1} */
} orc_log;

typedef struct {
    long nbox, nvar;     /* nvar = nsub*3*nbox */
    int nm;              /* number of modes */
    double *m, *a;       /* y_n */
    double *km[7], *ka[7];
    double *ym, *ya;     /* stage point */
    double mm7[128];
    int k1_valid, last_rejected;
    double t, dt;
    long n_attempts, n_accepted;
} orc_state;

/* ------------------------------------------------------------------------------------------- */
/* Dormand & Prince (1980) 5(4) tableau, as published (also Hairer, Norsett & Wanner I, Table   */
/* 5.2).  a[i][j] is the coupling of stage i+1 to slope j+1; b5 the 5th-order weights (equal to */
/* the 7th row: FSAL), b4 the embedded 4th-order weights.                                       */
/* ------------------------------------------------------------------------------------------- */
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84},
};
static const double DP_B5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784,
                                11.0 / 84, 0};
static const double DP_B4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

/* Exported so the tests can check the order conditions of the oracle's own tableau. */
void orc_tableau(double *a /*7*6*/, double *b5 /*7*/, double *b4 /*7*/)
{
    memcpy(a, DP_A, sizeof DP_A);
    memcpy(b5, DP_B5, sizeof DP_B5);
    memcpy(b4, DP_B4, sizeof DP_B4);
}

static int in_mask(const orc_problem *P, int x, int y, int z)
{
    if (x < 0 || y < 0 || z < 0 || x >= P->nx || y >= P->ny || z >= P->nz) return 0;
    return P->mask[x + (long)P->nx * (y + (long)P->ny * z)] != 0;
}

static long count_cells(const orc_problem *P)
{
    long nbox = (long)P->nx * P->ny * P->nz, n = 0;
    for (long i = 0; i < nbox; i++) n += P->mask[i] != 0;
    return n;
}

/* ------------------------------------------------------------------------------------------- */
/* Full magnetostatic demag.  The field of a uniformly magnetised cuboid cell j averaged over   */
/* cuboid cell i is -N(r_i - r_j) M_j with the cell-pair tensor of Newell, Williams & Dunlop    */
/* (1993): with D_h q(X) = 2 q(X) - q(X - h) - q(X + h) the negative second difference,          */
/*   N_xx(X, Y, Z) = D_dx D_dy D_dz f(X, Y, Z) / (4 pi dx dy dz),                                 */
/*   N_xy(X, Y, Z) = D_dx D_dy D_dz g(X, Y, Z) / (4 pi dx dy dz),                                 */
/* and the other components by permuting the axes.  B_d(r_i) = -mu0 Ms sum_j N(r_i - r_j) m_j,  */
/* summed over the magnetic cells directly (O(N_c^2), no FFT); for two sublattices m_j is the   */
/* total moment m1 + m2, as for the diagonal factors.                                           */
/* ------------------------------------------------------------------------------------------- */

/* Newell's f, even in every argument */
static double newell_f(double x, double y, double z)
{
    x = fabs(x);
    y = fabs(y);
    z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z, R = sqrt(x2 + y2 + z2);
    double t = (2.0 * x2 - y2 - z2) * R / 6.0;
    if (y > 0.0 && x2 + z2 > 0.0) t += 0.5 * y * (z2 - x2) * asinh(y / sqrt(x2 + z2));
    if (z > 0.0 && x2 + y2 > 0.0) t += 0.5 * z * (y2 - x2) * asinh(z / sqrt(x2 + y2));
    if (x > 0.0 && y > 0.0 && z > 0.0) t -= x * y * z * atan(y * z / (x * R));
    return t;
}

/* Newell's g, odd in x and in y, even in z */
static double newell_g(double x, double y, double z)
{
    const double sgn = (x < 0.0 ? -1.0 : 1.0) * (y < 0.0 ? -1.0 : 1.0);
    x = fabs(x);
    y = fabs(y);
    z = fabs(z);
    const double x2 = x * x, y2 = y * y, z2 = z * z, R = sqrt(x2 + y2 + z2);
    double t = -x * y * R / 3.0;
    if (z > 0.0 && x2 + y2 > 0.0) t += x * y * z * asinh(z / sqrt(x2 + y2));
    if (x > 0.0 && y2 + z2 > 0.0) t += y / 6.0 * (3.0 * z2 - y2) * asinh(x / sqrt(y2 + z2));
    if (y > 0.0 && x2 + z2 > 0.0) t += x / 6.0 * (3.0 * z2 - x2) * asinh(y / sqrt(x2 + z2));
    if (x > 0.0 && y > 0.0 && z > 0.0) {
        t -= z2 * z / 6.0 * atan(x * y / (z * R));
        t -= 0.5 * z * y2 * atan(x * z / (y * R));
        t -= 0.5 * z * x2 * atan(y * z / (x * R));
    }
    return sgn * t;
}

/* D_dx D_dy D_dz q(X, Y, Z) / (4 pi dx dy dz) for q = f (which = 0) or g (which = 1) */
static double newell_diff(int which, double X, double Y, double Z, double dx, double dy,
                          double dz)
{
    static const double w[3] = {-1.0, 2.0, -1.0};
    double s = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) {
                const double x = X + (i - 1) * dx, y = Y + (j - 1) * dy, z = Z + (k - 1) * dz;
                s += w[i] * w[j] * w[k] * (which ? newell_g(x, y, z) : newell_f(x, y, z));
            }
    return s / (4.0 * 3.14159265358979323846 * dx * dy * dz);
}

/* The cell-pair tensor of every displacement (X, Y, Z) = (i cx, j cy, k cz), |i| < nx,
   |j| < ny, |k| < nz: out[c * ND + ((k + nz - 1) * (2 ny - 1) + j + ny - 1) * (2 nx - 1) +
   i + nx - 1] with ND = (2nx-1)(2ny-1)(2nz-1) and components c = xx, yy, zz, xy, xz, yz. */
void orc_demag_tensor(int nx, int ny, int nz, double cx, double cy, double cz, double *out)
{
    const long Lx = 2L * nx - 1, Ly = 2L * ny - 1, Lz = 2L * nz - 1, ND = Lx * Ly * Lz;
#pragma omp parallel for schedule(dynamic)
    for (long k = 0; k < Lz; k++)
        for (long j = 0; j < Ly; j++)
            for (long i = 0; i < Lx; i++) {
                const double X = (double)(i - (nx - 1)) * cx, Y = (double)(j - (ny - 1)) * cy,
                             Z = (double)(k - (nz - 1)) * cz;
                const long o = (k * Ly + j) * Lx + i;
                out[0 * ND + o] = newell_diff(0, X, Y, Z, cx, cy, cz);
                out[1 * ND + o] = newell_diff(0, Y, X, Z, cy, cx, cz);
                out[2 * ND + o] = newell_diff(0, Z, Y, X, cz, cy, cx);
                out[3 * ND + o] = newell_diff(1, X, Y, Z, cx, cy, cz);
                out[4 * ND + o] = newell_diff(1, X, Z, Y, cx, cz, cy);
                out[5 * ND + o] = newell_diff(1, Y, Z, X, cy, cz, cx);
            }
}

/* Demag field of the total moment at every magnetic cell (dense box, 3 * nbox, zero outside
   the mask), by the direct sum over the magnetic cells. */
static void demag_field(const orc_problem *P, const double *m, double *bd)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz, ns = P->nsub;
    const long nbox = (long)nx * ny * nz;
    const long Lx = 2L * nx - 1, Ly = 2L * ny - 1, ND = Lx * Ly * (2L * nz - 1);
    const double dmg = ORC_MU0 * P->Ms;
#pragma omp parallel for schedule(dynamic)
    for (long ci = 0; ci < nbox; ci++) {
        bd[ci] = bd[nbox + ci] = bd[2 * nbox + ci] = 0.0;
        if (!P->mask[ci]) continue;
        const long xi = ci % nx, yi = (ci / nx) % ny, zi = ci / ((long)nx * ny);
        double h[3] = {0.0, 0.0, 0.0};
        for (long cj = 0; cj < nbox; cj++) {
            if (!P->mask[cj]) continue;
            const long xj = cj % nx, yj = (cj / nx) % ny, zj = cj / ((long)nx * ny);
            const long o = ((zi - zj + nz - 1) * Ly + (yi - yj + ny - 1)) * Lx + (xi - xj + nx - 1);
            double mj[3] = {0.0, 0.0, 0.0};
            for (int s = 0; s < ns; s++)
                for (int k = 0; k < 3; k++) mj[k] += m[(s * 3 + k) * nbox + cj];
            const double xx = P->demag[o], yy = P->demag[ND + o], zz = P->demag[2 * ND + o];
            const double xy = P->demag[3 * ND + o], xz = P->demag[4 * ND + o],
                         yz = P->demag[5 * ND + o];
            h[0] += xx * mj[0] + xy * mj[1] + xz * mj[2];
            h[1] += xy * mj[0] + yy * mj[1] + yz * mj[2];
            h[2] += xz * mj[0] + yz * mj[1] + zz * mj[2];
        }
        for (int k = 0; k < 3; k++) bd[k * nbox + ci] = -dmg * h[k];
    }
}

/* Exported for the tests: the full demag field (T) of the state m (dense box). */
int orc_demag_field(const orc_problem *P, const double *m, double *bd)
{
    if (!P->demag) return ORC_EINVAL;
    demag_field(P, m, bd);
    return ORC_OK;
}

/* Backward (feedback) coupling of mode n: gb~ if given, else the forward g~. */
static double gback_re(const orc_problem *P, int n) { return P->gb_re ? P->gb_re[n] : P->g_re[n]; }
static double gback_im(const orc_problem *P, int n) { return P->gb_im ? P->gb_im[n] : P->g_im[n]; }

static double profile(const orc_problem *P, int n, long cell)
{
    return P->u ? P->u[(long)n * P->nx * P->ny * P->nz + cell] : 1.0;
}

/*
 * Overlap <m^->_n = (1/N_c) sum_mask u_n (m_x - i m_y), Eq. (18) with Eq. (2).  For two
 * sublattices the cavity sees the net moment (m1 + m2)/2 (Sec. II G).
 */
void orc_overlap(const orc_problem *P, const double *m, double *mm)
{
    long nbox = (long)P->nx * P->ny * P->nz;
    double inv_nc = 1.0 / (double)count_cells(P);
    for (int n = 0; n < P->nmodes; n++) {
        double re = 0.0, im = 0.0;
        for (long c = 0; c < nbox; c++) {
            if (!P->mask[c]) continue;
            double mx = 0.0, my = 0.0;
            for (int s = 0; s < P->nsub; s++) {
                mx += m[(s * 3 + 0) * nbox + c];
                my += m[(s * 3 + 1) * nbox + c];
            }
            mx /= P->nsub;
            my /= P->nsub;
            double un = profile(P, n, c);
            re += un * mx;
            im -= un * my;
        }
        mm[2 * n] = re * inv_nc;
        mm[2 * n + 1] = im * inv_nc;
    }
}

/*
 * Right-hand side f(m, a) of the coupled system.  Writes dm (same layout as m; zero outside the
 * mask), da (2N) and the overlaps mm (2N).
 */
int orc_rhs(const orc_problem *P, const double *m, const double *a, double *dm, double *da,
            double *mm)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz, ns = P->nsub, N = P->nmodes;
    const long nbox = (long)nx * ny * nz;
    const double pre = -P->gamma / (1.0 + P->alpha * P->alpha);
    const double exch = 2.0 * P->Aex / P->Ms;           /* T m^2 */
    const double wx = exch / (P->cx * P->cx), wy = exch / (P->cy * P->cy),
                 wz = exch / (P->cz * P->cz);
    const double anis = 2.0 * P->Ku / P->Ms;            /* T */
    const double dmg = ORC_MU0 * P->Ms;                 /* T */
    /* Feedback amplitude of each mode: B_rf,x = sum_n u_n (2/gamma) Re[g~_n a_n]. */
    double hrf[64];
    if (N > 64 || ns < 1 || ns > 2) return ORC_EINVAL;
    for (int n = 0; n < N; n++) {
        double re_ga = gback_re(P, n) * a[2 * n] - gback_im(P, n) * a[2 * n + 1];
        hrf[n] = 2.0 / P->gamma * re_ga;
    }
    double *bd = NULL;   /* full demag field of the total moment */
    if (P->demag) {
        bd = malloc(3 * nbox * sizeof(double));
        if (!bd) return ORC_ENOMEM;
        demag_field(P, m, bd);
    }

#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; z++) {
        for (int y = 0; y < ny; y++) {
            for (int x = 0; x < nx; x++) {
                long c = x + (long)nx * (y + (long)ny * z);
                if (!P->mask[c]) {
                    for (int k = 0; k < 3 * ns; k++) dm[k * nbox + c] = 0.0;
                    continue;
                }
                double brf = 0.0;
                for (int n = 0; n < N; n++) brf += profile(P, n, c) * hrf[n];
                double mtot[3] = {0, 0, 0};
                for (int s = 0; s < ns; s++)
                    for (int k = 0; k < 3; k++) mtot[k] += m[(s * 3 + k) * nbox + c];
                for (int s = 0; s < ns; s++) {
                    const double *ms = m + (long)s * 3 * nbox;
                    double mi[3] = {ms[c], ms[nbox + c], ms[2 * nbox + c]};
                    double B[3] = {0, 0, 0};
                    /* exchange: sum over in-mask face neighbours of (m_j - m_i) / c_d^2 */
                    const int dx[6] = {-1, 1, 0, 0, 0, 0}, dy[6] = {0, 0, -1, 1, 0, 0},
                              dz[6] = {0, 0, 0, 0, -1, 1};
                    for (int q = 0; q < 6; q++) {
                        int xx = x + dx[q], yy = y + dy[q], zz = z + dz[q];
                        if (!in_mask(P, xx, yy, zz)) continue;
                        long j = xx + (long)nx * (yy + (long)ny * zz);
                        double w = dx[q] ? wx : (dy[q] ? wy : wz);
                        for (int k = 0; k < 3; k++) B[k] += w * (ms[k * nbox + j] - mi[k]);
                    }
                    /* uniaxial anisotropy (2 K_u / M_s)(m . k) k */
                    double mk = mi[0] * P->ku[0] + mi[1] * P->ku[1] + mi[2] * P->ku[2];
                    for (int k = 0; k < 3; k++) B[k] += anis * mk * P->ku[k];
                    /* Zeeman and demag of the total moment (diagonal factors or full) */
                    for (int k = 0; k < 3; k++)
                        B[k] += P->B0[k] + (bd ? bd[k * nbox + c] : -dmg * P->Nd[k] * mtot[k]);
                    /* inter-sublattice exchange field */
                    if (ns == 2) {
                        const double *mo = m + (long)(1 - s) * 3 * nbox;
                        for (int k = 0; k < 3; k++) B[k] -= P->BE * mo[k * nbox + c];
                    }
                    /* cavity feedback along x */
                    B[0] += brf;
                    /* Landau-Lifshitz-Gilbert torque */
                    double t1[3] = {mi[1] * B[2] - mi[2] * B[1], mi[2] * B[0] - mi[0] * B[2],
                                    mi[0] * B[1] - mi[1] * B[0]};
                    double t2[3] = {mi[1] * t1[2] - mi[2] * t1[1], mi[2] * t1[0] - mi[0] * t1[2],
                                    mi[0] * t1[1] - mi[1] * t1[0]};
                    for (int k = 0; k < 3; k++)
                        dm[(s * 3 + k) * nbox + c] = pre * (t1[k] + P->alpha * t2[k]);
                }
            }
        }
    }

    free(bd);
    orc_overlap(P, m, mm);
    for (int n = 0; n < N; n++) {
        double ar = a[2 * n], ai = a[2 * n + 1];
        /* (-i w - kappa) a */
        double r = -P->kappa[n] * ar + P->omega[n] * ai;
        double i = -P->kappa[n] * ai - P->omega[n] * ar;
        /* + i g~ <m^-> = i (g_re + i g_im)(mr + i mi) */
        double gr = P->g_re[n], gi = P->g_im[n], mr = mm[2 * n], mi = mm[2 * n + 1];
        double pr = gr * mr - gi * mi, pi = gr * mi + gi * mr; /* g~ <m^-> */
        r += -pi;
        i += pr;
        /* self-Kerr -i K |a|^2 a */
        if (P->kerr) {
            const double k2 = P->kerr[n] * (ar * ar + ai * ai);
            r += k2 * ai;
            i -= k2 * ar;
        }
        da[2 * n] = P->cavity_frozen ? 0.0 : r;
        da[2 * n + 1] = P->cavity_frozen ? 0.0 : i;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------- */
/* integrator state                                                                            */
/* ------------------------------------------------------------------------------------------- */
void orc_state_free(orc_state *S)
{
    if (!S) return;
    free(S->m);
    free(S->a);
    free(S->ym);
    free(S->ya);
    for (int j = 0; j < 7; j++) {
        free(S->km[j]);
        free(S->ka[j]);
    }
    free(S);
}

orc_state *orc_state_new(const orc_problem *P)
{
    orc_state *S = calloc(1, sizeof *S);
    if (!S) return NULL;
    S->nbox = (long)P->nx * P->ny * P->nz;
    S->nvar = (long)P->nsub * 3 * S->nbox;
    S->nm = P->nmodes;
    long na = 2 * (long)(P->nmodes > 0 ? P->nmodes : 1);
    S->m = calloc(S->nvar, sizeof(double));
    S->ym = calloc(S->nvar, sizeof(double));
    S->a = calloc(na, sizeof(double));
    S->ya = calloc(na, sizeof(double));
    int ok = S->m && S->ym && S->a && S->ya;
    for (int j = 0; j < 7; j++) {
        S->km[j] = calloc(S->nvar, sizeof(double));
        S->ka[j] = calloc(na, sizeof(double));
        ok = ok && S->km[j] && S->ka[j];
    }
    if (!ok) {
        orc_state_free(S);
        return NULL;
    }
    return S;
}

void orc_state_set(orc_state *S, const double *m, const double *a, double t, double dt)
{
    memcpy(S->m, m, S->nvar * sizeof(double));
    memcpy(S->a, a, 2 * S->nm * sizeof(double));
    S->t = t;
    S->dt = dt;
    S->k1_valid = 0;
    S->last_rejected = 0;
    S->n_attempts = S->n_accepted = 0;
}

void orc_state_get(const orc_state *S, double *m, double *a, double *t, double *dt,
                   long *counts /*2: attempts, accepted*/)
{
    if (m) memcpy(m, S->m, S->nvar * sizeof(double));
    if (a) memcpy(a, S->a, 2 * S->nm * sizeof(double));
    if (t) *t = S->t;
    if (dt) *dt = S->dt;
    if (counts) {
        counts[0] = S->n_attempts;
        counts[1] = S->n_accepted;
    }
}

/* The drive at time t added to the cavity slopes da (Eq. (1), (12)). */
static void add_drive(const orc_problem *P, double t, double *da)
{
    if (!P->drive_re || P->cavity_frozen) return;
    const double x = (t - P->drive_t0) / P->drive_sigma;
    const double env = exp(-0.5 * x * x);
    for (int n = 0; n < P->nmodes; n++) {
        da[2 * n] += P->drive_re[n] * env;
        da[2 * n + 1] += P->drive_im[n] * env;
    }
}

/* Pump coefficient Q_n(t) = P_n e^{-i wp_n t} of the parametric term. */
static void pump_coefficient(const orc_problem *P, int n, double t, double *qr, double *qi)
{
    const double c = cos(P->pump_w[n] * t), s = sin(P->pump_w[n] * t);
    *qr = P->pump_re[n] * c + P->pump_im[n] * s;
    *qi = P->pump_im[n] * c - P->pump_re[n] * s;
}

/* The parametric term at time t, -i Q_n(t) conj(a_n), added to the cavity slopes da:
   -i (qr + i qi)(ar - i ai) = (qi ar - qr ai) - i (qr ar + qi ai). */
static void add_pump(const orc_problem *P, double t, const double *a, double *da)
{
    if (!P->pump_re || P->cavity_frozen) return;
    for (int n = 0; n < P->nmodes; n++) {
        double qr, qi;
        pump_coefficient(P, n, t, &qr, &qi);
        const double ar = a[2 * n], ai = a[2 * n + 1];
        da[2 * n] += qi * ar - qr * ai;
        da[2 * n + 1] -= qr * ar + qi * ai;
    }
}

/* Node c_s of stage s (0-based) of the tableau: the row sum of its couplings. */
static double dp_node(int s)
{
    double c = 0.0;
    for (int j = 0; j < 6; j++) c += DP_A[s][j];
    return c;
}

/*
 * One Dormand-Prince attempt of size h from (S->m, S->a).  On return the 5th-order point y7 is
 * in (S->ym, S->ya), its slope in km[6]/ka[6] and the scaled error in *err.
 */
static int dp_attempt(const orc_problem *P, orc_state *S, const orc_solver *sv, double h,
                      double *err)
{
    const long nv = S->nvar, nbox = S->nbox;
    const int N = S->nm;
    double mm[128];
    if (!S->k1_valid) {
        int rc = orc_rhs(P, S->m, S->a, S->km[0], S->ka[0], mm);
        if (rc) return rc;
        add_drive(P, S->t, S->ka[0]);
        add_pump(P, S->t, S->a, S->ka[0]);
        S->k1_valid = 1;
    }
    for (int s = 1; s < 7; s++) {
        /* stage point y_s = y_n + h sum_{j<s} a_sj k_j */
        for (long i = 0; i < nv; i++) {
            double acc = S->m[i];
            for (int j = 0; j < s; j++) acc += h * DP_A[s][j] * S->km[j][i];
            S->ym[i] = acc;
        }
        for (int i = 0; i < 2 * N; i++) {
            double acc = S->a[i];
            for (int j = 0; j < s; j++) acc += h * DP_A[s][j] * S->ka[j][i];
            S->ya[i] = acc;
        }
        int rc = orc_rhs(P, S->ym, S->ya, S->km[s], S->ka[s], mm);
        if (rc) return rc;
        add_drive(P, S->t + dp_node(s) * h, S->ka[s]);
        add_pump(P, S->t + dp_node(s) * h, S->ya, S->ka[s]);
    }
    memcpy(S->mm7, mm, 2 * N * sizeof(double));

    /* error estimate e = h sum_j (b5_j - b4_j) k_j, taken from the slopes directly */
    double em = 0.0;
    for (int s = 0; s < P->nsub; s++)
        for (int k = 0; k < 3; k++)
            for (long c = 0; c < nbox; c++) {
                if (!P->mask[c]) continue;
                long i = (s * 3 + k) * nbox + c;
                double e = 0.0;
                for (int j = 0; j < 7; j++) e += (DP_B5[j] - DP_B4[j]) * S->km[j][i];
                e = fabs(h * e);
                if (e > em || isnan(e)) em = e;
            }
    double ea = 0.0, amax = 0.0;
    for (int n = 0; n < N; n++) {
        double er = 0.0, ei = 0.0;
        for (int j = 0; j < 7; j++) {
            er += (DP_B5[j] - DP_B4[j]) * S->ka[j][2 * n];
            ei += (DP_B5[j] - DP_B4[j]) * S->ka[j][2 * n + 1];
        }
        double e = fabs(h) * sqrt(er * er + ei * ei);
        if (e > ea || isnan(e)) ea = e;
        double a0 = hypot(S->a[2 * n], S->a[2 * n + 1]);
        double a1 = hypot(S->ya[2 * n], S->ya[2 * n + 1]);
        if (a0 > amax) amax = a0;
        if (a1 > amax) amax = a1;
    }
    double scale_a = sv->rtol * (amax > sv->a_ref ? amax : sv->a_ref);
    double e1 = em / sv->rtol, e2 = ea / scale_a;
    *err = (e1 > e2 || isnan(e1)) ? e1 : e2;
    if (isnan(*err)) return ORC_ENAN;
    return ORC_OK;
}

/* Accept the attempt held in S: y_{n+1} = y7 with m renormalised per cell; FSAL k1 <- k7. */
static void dp_accept(const orc_problem *P, orc_state *S, double h)
{
    const long nbox = S->nbox;
    for (int s = 0; s < P->nsub; s++)
        for (long c = 0; c < nbox; c++) {
            double *x = S->ym + (s * 3 + 0) * nbox + c, *y = x + nbox, *z = y + nbox;
            if (!P->mask[c]) {
                *x = *y = *z = 0.0;
                continue;
            }
            double r = sqrt(*x * *x + *y * *y + *z * *z);
            *x /= r;
            *y /= r;
            *z /= r;
        }
    double *tm = S->m;
    S->m = S->ym;
    S->ym = tm;
    double *ta = S->a;
    S->a = S->ya;
    S->ya = ta;
    double *k = S->km[0];
    S->km[0] = S->km[6];
    S->km[6] = k;
    k = S->ka[0];
    S->ka[0] = S->ka[6];
    S->ka[6] = k;
    S->t += h;
    S->n_accepted++;
}

static void log_attempt(orc_log *L, const orc_state *S, double t, double h, double err, int acc)
{
    if (!L || L->n >= L->cap) {
        if (L) L->n++;
        return;
    }
    int i = L->n++;
    L->t[i] = t;
    L->dt[i] = h;
    L->err[i] = err;
    L->accepted[i] = acc;
    for (int q = 0; q < 2 * S->nm; q++) {
        if (L->a) L->a[(long)i * 2 * S->nm + q] = S->a[q];
        if (L->mm) L->mm[(long)i * 2 * S->nm + q] = S->mm7[q];
    }
}

/*
 * Adaptive integration from S->t to T.  Step-size rule: err <= 1 accepts;
 * factor = clamp(0.9 err^(-1/5), 0.2, 5) (5 when err = 0), capped at 1 right after a rejection;
 * the next step is min(h * factor, dt_max); an attempt that would pass T is shortened to land on
 * T exactly.  Stops after max_attempts attempts.
 */
int orc_run(const orc_problem *P, orc_state *S, const orc_solver *sv, double T,
            long max_attempts, orc_log *L)
{
    long n = 0;
    while (S->t < T && n < max_attempts) {
        double h = S->dt;
        if (h > sv->dt_max) h = sv->dt_max;
        int last = 0;
        if (S->t + h >= T) {
            h = T - S->t;
            last = 1;
        }
        double err;
        int rc = dp_attempt(P, S, sv, h, &err);
        S->n_attempts++;
        n++;
        if (rc) return rc;
        double fac = (err > 0.0) ? 0.9 * pow(err, -0.2) : 5.0;
        if (fac > 5.0) fac = 5.0;
        if (fac < 0.2) fac = 0.2;
        if (err <= 1.0) {
            if (S->last_rejected && fac > 1.0) fac = 1.0;
            dp_accept(P, S, h);
            if (last) S->t = T;
            log_attempt(L, S, S->t, h, err, 1);
            S->last_rejected = 0;
            double hn = h * fac;
            S->dt = hn > sv->dt_max ? sv->dt_max : hn;
        } else {
            log_attempt(L, S, S->t, h, err, 0);
            S->last_rejected = 1;
            S->dt = h * fac;
            if (S->dt < sv->dt_min) return ORC_ESTEPFAIL;
        }
    }
    return ORC_OK;
}

/* Replay: take exactly the given step sizes, every step accepted (for parity checks). */
int orc_replay(const orc_problem *P, orc_state *S, const orc_solver *sv, const double *dts,
               long n, orc_log *L)
{
    for (long i = 0; i < n; i++) {
        double err;
        int rc = dp_attempt(P, S, sv, dts[i], &err);
        S->n_attempts++;
        if (rc) return rc;
        dp_accept(P, S, dts[i]);
        log_attempt(L, S, S->t, dts[i], err, 1);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------- */
/* Discrete adjoint (reverse mode) of a replayed Dormand-Prince step sequence.                  */
/* Not in the paper: it differentiates exactly the computation above (stages, FSAL slope taken  */
/* at the un-normalised 5th-order point, renormalisation of m on accept) with the step sizes     */
/* held fixed.                                                                                  */
/* ------------------------------------------------------------------------------------------- */

/* Parameter gradients; every pointer may be NULL.  The routines below ADD into them. */
typedef struct {
    double *g_re, *g_im, *kappa, *omega; /* nmodes each: dL/d Re g~_n, dL/d Im g~_n, ... */
    double *alpha;                       /* 1 */
    double *u;                           /* nmodes * nbox (only with profiles) */
    double *gb_re, *gb_im;               /* nmodes each, with nonreciprocal coupling */
    double *kerr;                        /* nmodes, with a Kerr term */
    double *pump_re, *pump_im;           /* nmodes each, with a parametric pump: dL/d Re P_n, ... */
} orc_grads;

/*
 * Transpose of the parametric term at time t (see add_pump): the slope (qi ar - qr ai,
 * -qr ar - qi ai) has the symmetric Jacobian [[qi, -qr], [-qr, -qi]] in (ar, ai), so ga gets
 * (qi wr - qr wi, -qr wr - qi wi); with d(qr, qi)/d(Pr) = (c, -s) and d(qr, qi)/d(Pi) = (s, c),
 * c = cos(wp t), s = sin(wp t), the pump gradients follow from dL/dqr = -ai wr - ar wi and
 * dL/dqi = ar wr - ai wi.
 */
static void pump_vjp(const orc_problem *P, double t, const double *a, const double *wa,
                     double *ga, orc_grads *G)
{
    if (!P->pump_re || P->cavity_frozen) return;
    for (int n = 0; n < P->nmodes; n++) {
        double qr, qi;
        pump_coefficient(P, n, t, &qr, &qi);
        const double ar = a[2 * n], ai = a[2 * n + 1], wr = wa[2 * n], wi = wa[2 * n + 1];
        ga[2 * n] += qi * wr - qr * wi;
        ga[2 * n + 1] += -qr * wr - qi * wi;
        const double lqr = -ai * wr - ar * wi, lqi = ar * wr - ai * wi;
        const double c = cos(P->pump_w[n] * t), sn = sin(P->pump_w[n] * t);
        if (G && G->pump_re) G->pump_re[n] += lqr * c - lqi * sn;
        if (G && G->pump_im) G->pump_im[n] += lqr * sn + lqi * c;
    }
}

/*
 * Vector-Jacobian product of orc_rhs at (m, a).  Given adjoint weights wm (layout of m) on the
 * slopes dm and wa (2N) on da, ADDS (df/dm)^T w to gm, (df/da)^T w to ga and (df/dtheta)^T w to
 * the parameter gradients.  Each term of the forward evaluation is transposed on its own, in
 * scatter form: the forward adds w_d (m_j - m_i) to B_i for every in-mask neighbour j, so its
 * transpose adds w_d Bbar_i to gm_j and subtracts it from gm_i.
 */
int orc_rhs_vjp(const orc_problem *P, const double *m, const double *a, const double *wm,
                const double *wa, double *gm, double *ga, orc_grads *G)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz, ns = P->nsub, N = P->nmodes;
    const long nbox = (long)nx * ny * nz;
    const double opa = 1.0 + P->alpha * P->alpha;
    const double pre = -P->gamma / opa;
    const double exch = 2.0 * P->Aex / P->Ms;
    const double wx = exch / (P->cx * P->cx), wy = exch / (P->cy * P->cy),
                 wz = exch / (P->cz * P->cz);
    const double anis = 2.0 * P->Ku / P->Ms;
    const double dmg = ORC_MU0 * P->Ms;
    if (N > 64 || ns < 1 || ns > 2) return ORC_EINVAL;
    if (P->demag) return ORC_EINVAL;   /* the adjoint covers the diagonal demag factors only */
    const int want_u = P->u && G && G->u;
    double hrf[64], hbar[64], mm[128];
    for (int n = 0; n < N; n++) {
        hrf[n] = 2.0 / P->gamma * (gback_re(P, n) * a[2 * n] - gback_im(P, n) * a[2 * n + 1]);
        hbar[n] = 0.0;
    }
    orc_overlap(P, m, mm);
    double *Bb = calloc((size_t)ns * 3 * nbox, sizeof(double));
    if (!Bb) return ORC_ENOMEM;
    const int dx[6] = {-1, 1, 0, 0, 0, 0}, dy[6] = {0, 0, -1, 1, 0, 0}, dz[6] = {0, 0, 0, 0, -1, 1};

    /* pass 1: the field B of every cell (as in orc_rhs), the torque's local transpose and the
       adjoint of the field, Bbar = (dT/dB)^T w */
    double galpha = 0.0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long c = x + (long)nx * (y + (long)ny * z);
                if (!P->mask[c]) continue;
                double brf = 0.0;
                for (int n = 0; n < N; n++) brf += profile(P, n, c) * hrf[n];
                double mtot[3] = {0, 0, 0};
                for (int s = 0; s < ns; s++)
                    for (int k = 0; k < 3; k++) mtot[k] += m[(s * 3 + k) * nbox + c];
                for (int s = 0; s < ns; s++) {
                    const double *ms = m + (long)s * 3 * nbox;
                    double mi[3] = {ms[c], ms[nbox + c], ms[2 * nbox + c]};
                    double B[3] = {0, 0, 0};
                    for (int q = 0; q < 6; q++) {
                        int xx = x + dx[q], yy = y + dy[q], zz = z + dz[q];
                        if (!in_mask(P, xx, yy, zz)) continue;
                        long j = xx + (long)nx * (yy + (long)ny * zz);
                        double w = dx[q] ? wx : (dy[q] ? wy : wz);
                        for (int k = 0; k < 3; k++) B[k] += w * (ms[k * nbox + j] - mi[k]);
                    }
                    double mk = mi[0] * P->ku[0] + mi[1] * P->ku[1] + mi[2] * P->ku[2];
                    for (int k = 0; k < 3; k++) B[k] += anis * mk * P->ku[k];
                    for (int k = 0; k < 3; k++) B[k] += P->B0[k] - dmg * P->Nd[k] * mtot[k];
                    if (ns == 2) {
                        const double *mo = m + (long)(1 - s) * 3 * nbox;
                        for (int k = 0; k < 3; k++) B[k] -= P->BE * mo[k * nbox + c];
                    }
                    B[0] += brf;
                    double w[3];
                    for (int k = 0; k < 3; k++) w[k] = wm[(s * 3 + k) * nbox + c];
                    /* T = pre (T1 + alpha T2), T1 = m x B, T2 = m x T1 = m (m.B) - B (m.m) */
                    double T1[3] = {mi[1] * B[2] - mi[2] * B[1], mi[2] * B[0] - mi[0] * B[2],
                                    mi[0] * B[1] - mi[1] * B[0]};
                    double T2[3] = {mi[1] * T1[2] - mi[2] * T1[1], mi[2] * T1[0] - mi[0] * T1[2],
                                    mi[0] * T1[1] - mi[1] * T1[0]};
                    double mB = mi[0] * B[0] + mi[1] * B[1] + mi[2] * B[2];
                    double wmi = w[0] * mi[0] + w[1] * mi[1] + w[2] * mi[2];
                    double wB = w[0] * B[0] + w[1] * B[1] + w[2] * B[2];
                    double mmi = mi[0] * mi[0] + mi[1] * mi[1] + mi[2] * mi[2];
                    /* w . T1 = m . (B x w)  ->  d/dm = B x w,  d/dB = w x m */
                    double Bxw[3] = {B[1] * w[2] - B[2] * w[1], B[2] * w[0] - B[0] * w[2],
                                     B[0] * w[1] - B[1] * w[0]};
                    /* w . T2 = (w.m)(m.B) - (w.B)(m.m) */
                    for (int k = 0; k < 3; k++) {
                        double dT2dm = w[k] * mB + wmi * B[k] - 2.0 * wB * mi[k];
                        double dT2dB = wmi * mi[k] - mmi * w[k];
                        gm[(s * 3 + k) * nbox + c] += pre * (Bxw[k] + P->alpha * dT2dm);
                        Bb[(s * 3 + k) * nbox + c] = pre * P->alpha * dT2dB;
                    }
                    double wxm[3] = {w[1] * mi[2] - w[2] * mi[1], w[2] * mi[0] - w[0] * mi[2],
                                     w[0] * mi[1] - w[1] * mi[0]};
                    for (int k = 0; k < 3; k++) Bb[(s * 3 + k) * nbox + c] += pre * wxm[k];
                    /* d pre / d alpha = -pre 2 alpha / (1 + alpha^2) */
                    for (int k = 0; k < 3; k++) {
                        double Tk = pre * (T1[k] + P->alpha * T2[k]);
                        galpha += w[k] * (-2.0 * P->alpha / opa * Tk + pre * T2[k]);
                    }
                }
            }

    /* pass 2: transpose of the field B(m, a) */
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long c = x + (long)nx * (y + (long)ny * z);
                if (!P->mask[c]) continue;
                for (int s = 0; s < ns; s++) {
                    double bb[3];
                    for (int k = 0; k < 3; k++) bb[k] = Bb[(s * 3 + k) * nbox + c];
                    double *g = gm + (long)s * 3 * nbox;
                    /* exchange */
                    for (int q = 0; q < 6; q++) {
                        int xx = x + dx[q], yy = y + dy[q], zz = z + dz[q];
                        if (!in_mask(P, xx, yy, zz)) continue;
                        long j = xx + (long)nx * (yy + (long)ny * zz);
                        double w = dx[q] ? wx : (dy[q] ? wy : wz);
                        for (int k = 0; k < 3; k++) {
                            g[k * nbox + j] += w * bb[k];
                            g[k * nbox + c] -= w * bb[k];
                        }
                    }
                    /* anisotropy */
                    double bk = bb[0] * P->ku[0] + bb[1] * P->ku[1] + bb[2] * P->ku[2];
                    for (int k = 0; k < 3; k++) g[k * nbox + c] += anis * bk * P->ku[k];
                    /* demag of the total moment: every sublattice */
                    for (int s2 = 0; s2 < ns; s2++)
                        for (int k = 0; k < 3; k++)
                            gm[(s2 * 3 + k) * nbox + c] -= dmg * P->Nd[k] * bb[k];
                    /* inter-sublattice exchange */
                    if (ns == 2)
                        for (int k = 0; k < 3; k++)
                            gm[((1 - s) * 3 + k) * nbox + c] -= P->BE * bb[k];
                    /* feedback B_x += sum_n u_n hrf_n */
                    for (int n = 0; n < N; n++) {
                        hbar[n] += profile(P, n, c) * bb[0];
                        if (want_u) G->u[(long)n * nbox + c] += hrf[n] * bb[0];
                    }
                }
            }
    free(Bb);
    if (G && G->alpha) *G->alpha += galpha;

    /* hrf_n = (2/gamma) (Re gb~ Re a - Im gb~ Im a); with reciprocal coupling gb~ is g~ and its
       gradient goes to g~, otherwise to gb~ */
    for (int n = 0; n < N; n++) {
        const double c2 = 2.0 / P->gamma * hbar[n];
        ga[2 * n] += c2 * gback_re(P, n);
        ga[2 * n + 1] -= c2 * gback_im(P, n);
        double *dre = P->gb_re ? (G ? G->gb_re : NULL) : (G ? G->g_re : NULL);
        double *dim = P->gb_re ? (G ? G->gb_im : NULL) : (G ? G->g_im : NULL);
        if (dre) dre[n] += c2 * a[2 * n];
        if (dim) dim[n] -= c2 * a[2 * n + 1];
    }

    /* cavity slopes: da_re = -k ar + w ai - (gr mi + gi mr), da_im = -k ai - w ar + (gr mr - gi mi) */
    const double inv = 1.0 / ((double)count_cells(P) * ns);
    for (int n = 0; n < N; n++) {
        const double wr = wa[2 * n], wi = wa[2 * n + 1];
        const double ar = a[2 * n], ai = a[2 * n + 1];
        const double gr = P->g_re[n], gi = P->g_im[n], mr = mm[2 * n], mi = mm[2 * n + 1];
        ga[2 * n] += -P->kappa[n] * wr - P->omega[n] * wi;
        ga[2 * n + 1] += P->omega[n] * wr - P->kappa[n] * wi;
        if (P->kerr) {   /* -i K |a|^2 a: (K|a|^2 ai, -K|a|^2 ar) */
            const double K = P->kerr[n], s2 = ar * ar + ai * ai;
            ga[2 * n] += wr * 2.0 * K * ar * ai - wi * K * (3.0 * ar * ar + ai * ai);
            ga[2 * n + 1] += wr * K * (ar * ar + 3.0 * ai * ai) - wi * 2.0 * K * ar * ai;
            if (G && G->kerr) G->kerr[n] += s2 * (wr * ai - wi * ar);
        }
        if (G && G->g_re) G->g_re[n] += -mi * wr + mr * wi;
        if (G && G->g_im) G->g_im[n] += -mr * wr - mi * wi;
        if (G && G->kappa) G->kappa[n] += -ar * wr - ai * wi;
        if (G && G->omega) G->omega[n] += ai * wr - ar * wi;
        const double mbr = -gi * wr + gr * wi, mbi = -gr * wr - gi * wi;
        /* overlap: mm_re = inv sum u sum_s m_x, mm_im = -inv sum u sum_s m_y */
        for (long c = 0; c < nbox; c++) {
            if (!P->mask[c]) continue;
            const double un = profile(P, n, c);
            double sx = 0.0, sy = 0.0;
            for (int s = 0; s < ns; s++) {
                gm[(s * 3 + 0) * nbox + c] += inv * un * mbr;
                gm[(s * 3 + 1) * nbox + c] -= inv * un * mbi;
                sx += m[(s * 3 + 0) * nbox + c];
                sy += m[(s * 3 + 1) * nbox + c];
            }
            if (want_u) G->u[(long)n * nbox + c] += inv * (mbr * sx - mbi * sy);
        }
    }
    return ORC_OK;
}

/*
 * Gradient of a loss L(a_0, ..., a_n, m_n) through n replayed steps of sizes dts from (m0, a0)
 * (the states a_i after i steps; y_0 = (m0, a0) as given, not renormalised).
 * dL_da: (n+1) x 2N, row i = dL/d a_i (NULL: zero); dL_dm: dL/d m_n (NULL: zero).
 * Writes dL/d m0 (gm0, nvar) and dL/d a0 (ga0, 2N) and ADDS the parameter gradients to G.
 * The state (m_i, a_i) and the FSAL slope k1_i of every step are kept; the reverse sweep
 * recomputes the stages of step i from them and runs through the stages last to first:
 *   stage point Y_s = y_i + h sum_{j<s} A_sj k_j,  k_s = f(Y_s) (s = 2..7; k_1 given),
 *   y_{i+1} = (normalise(Y_7,m), Y_7,a),  k1_{i+1} = k_7.
 * With F_s the adjoint of Y_s: F_7 = J_norm(Y_7)^T ybar_{i+1} + J_f(Y_7)^T k1bar_{i+1},
 * F_s = J_f(Y_s)^T (h sum_{s'>s} A_s's F_s') for s = 6..2, and then
 * ybar_i = sum_s F_s, k1bar_i = h sum_s A_s1 F_s.  Step 0's slope k1 = f(y_0) adds
 * J_f(y_0)^T k1bar_0 at the end.
 */
int orc_adjoint(const orc_problem *P, const orc_solver *sv, const double *m0, const double *a0,
                const double *dts, long n, const double *dL_da, const double *dL_dm,
                double *gm0, double *ga0, orc_grads *G, double t_start)
{
    orc_state *S = orc_state_new(P);
    if (!S) return ORC_ENOMEM;
    const long nv = S->nvar, nbox = S->nbox;
    const int N = P->nmodes, na = 2 * (N > 0 ? N : 1), ns = P->nsub;
    int rc = ORC_OK;
    double *Mst = malloc((size_t)(n > 0 ? n : 1) * nv * sizeof(double));
    double *Kst = malloc((size_t)(n > 0 ? n : 1) * nv * sizeof(double));
    double *Ast = malloc((size_t)(n > 0 ? n : 1) * na * sizeof(double));
    double *KAst = malloc((size_t)(n > 0 ? n : 1) * na * sizeof(double));
    double *Tst = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *Ym[7], *Ya[7], *Fm[7], *Fa[7];
    double *lm = calloc(nv, sizeof(double)), *la = calloc(na, sizeof(double));
    double *lkm = calloc(nv, sizeof(double)), *lka = calloc(na, sizeof(double));
    double *wkm = calloc(nv, sizeof(double)), *wka = calloc(na, sizeof(double));
    int ok = Mst && Kst && Ast && KAst && Tst && lm && la && lkm && lka && wkm && wka;
    for (int s = 0; s < 7; s++) {
        Ym[s] = calloc(nv, sizeof(double));
        Fm[s] = calloc(nv, sizeof(double));
        Ya[s] = calloc(na, sizeof(double));
        Fa[s] = calloc(na, sizeof(double));
        ok = ok && Ym[s] && Fm[s] && Ya[s] && Fa[s];
    }
    if (!ok) {
        rc = ORC_ENOMEM;
        goto done;
    }

    /* forward: keep (m_i, a_i, k1_i) of every step */
    orc_state_set(S, m0, a0, t_start, n > 0 ? dts[0] : 1.0);
    for (long i = 0; i < n; i++) {
        double err;
        Tst[i] = S->t;
        memcpy(Mst + i * nv, S->m, nv * sizeof(double));
        memcpy(Ast + i * na, S->a, 2 * N * sizeof(double));
        rc = dp_attempt(P, S, sv, dts[i], &err);
        if (rc) goto done;
        memcpy(Kst + i * nv, S->km[0], nv * sizeof(double));
        memcpy(KAst + i * na, S->ka[0], 2 * N * sizeof(double));
        dp_accept(P, S, dts[i]);
    }

    /* reverse */
    if (dL_dm) memcpy(lm, dL_dm, nv * sizeof(double));
    if (dL_da) memcpy(la, dL_da + n * 2 * N, 2 * N * sizeof(double));
    for (long i = n - 1; i >= 0; i--) {
        const double h = dts[i];
        double err;
        memcpy(S->m, Mst + i * nv, nv * sizeof(double));
        memcpy(S->a, Ast + i * na, 2 * N * sizeof(double));
        memcpy(S->km[0], Kst + i * nv, nv * sizeof(double));
        memcpy(S->ka[0], KAst + i * na, 2 * N * sizeof(double));
        S->t = Tst[i];
        S->k1_valid = 1;
        rc = dp_attempt(P, S, sv, h, &err);
        if (rc) goto done;
        /* stage points of stages 2..7 (0-based 1..6) */
        for (int s = 1; s < 7; s++) {
            for (long v = 0; v < nv; v++) {
                double acc = S->m[v];
                for (int j = 0; j < s; j++) acc += h * DP_A[s][j] * S->km[j][v];
                Ym[s][v] = acc;
            }
            for (int q = 0; q < 2 * N; q++) {
                double acc = S->a[q];
                for (int j = 0; j < s; j++) acc += h * DP_A[s][j] * S->ka[j][q];
                Ya[s][q] = acc;
            }
            memset(Fm[s], 0, nv * sizeof(double));
            memset(Fa[s], 0, na * sizeof(double));
        }
        /* stage 7: renormalisation of m, direct a, and the FSAL slope k1_{i+1} = k_7 */
        for (int s = 0; s < ns; s++)
            for (long c = 0; c < nbox; c++) {
                if (!P->mask[c]) continue;
                double y[3], l[3];
                for (int k = 0; k < 3; k++) {
                    y[k] = Ym[6][(s * 3 + k) * nbox + c];
                    l[k] = lm[(s * 3 + k) * nbox + c];
                }
                const double r = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
                const double nl = (y[0] * l[0] + y[1] * l[1] + y[2] * l[2]) / r;
                for (int k = 0; k < 3; k++) Fm[6][(s * 3 + k) * nbox + c] = (l[k] - y[k] / r * nl) / r;
            }
        for (int q = 0; q < 2 * N; q++) Fa[6][q] = la[q];
        rc = orc_rhs_vjp(P, Ym[6], Ya[6], lkm, lka, Fm[6], Fa[6], G);
        if (rc) goto done;
        pump_vjp(P, Tst[i] + dp_node(6) * h, Ya[6], lka, Fa[6], G);
        for (int s = 5; s >= 1; s--) {
            for (long v = 0; v < nv; v++) {
                double acc = 0.0;
                for (int t = s + 1; t < 7; t++) acc += h * DP_A[t][s] * Fm[t][v];
                wkm[v] = acc;
            }
            for (int q = 0; q < 2 * N; q++) {
                double acc = 0.0;
                for (int t = s + 1; t < 7; t++) acc += h * DP_A[t][s] * Fa[t][q];
                wka[q] = acc;
            }
            rc = orc_rhs_vjp(P, Ym[s], Ya[s], wkm, wka, Fm[s], Fa[s], G);
            if (rc) goto done;
            pump_vjp(P, Tst[i] + dp_node(s) * h, Ya[s], wka, Fa[s], G);
        }
        for (long v = 0; v < nv; v++) {
            double sy = 0.0, sk = 0.0;
            for (int s = 1; s < 7; s++) {
                sy += Fm[s][v];
                sk += h * DP_A[s][0] * Fm[s][v];
            }
            lm[v] = sy;
            lkm[v] = sk;
        }
        for (int q = 0; q < 2 * N; q++) {
            double sy = 0.0, sk = 0.0;
            for (int s = 1; s < 7; s++) {
                sy += Fa[s][q];
                sk += h * DP_A[s][0] * Fa[s][q];
            }
            la[q] = sy + (dL_da ? dL_da[i * 2 * N + q] : 0.0);
            lka[q] = sk;
        }
    }
    if (n == 0 && dL_da)
        for (int q = 0; q < 2 * N; q++) la[q] = dL_da[q];
    /* step 0 evaluated its first slope at y_0 */
    if (n > 0) {
        rc = orc_rhs_vjp(P, m0, a0, lkm, lka, lm, la, G);
        if (rc) goto done;
        pump_vjp(P, Tst[0], a0, lka, la, G);
    }
    if (gm0) memcpy(gm0, lm, nv * sizeof(double));
    if (ga0) memcpy(ga0, la, 2 * N * sizeof(double));

done:
    free(Mst);
    free(Kst);
    free(Ast);
    free(KAst);
    free(Tst);
    free(lm);
    free(la);
    free(lkm);
    free(lka);
    free(wkm);
    free(wka);
    for (int s = 0; s < 7; s++) {
        free(Ym[s]);
        free(Ya[s]);
        free(Fm[s]);
        free(Fa[s]);
    }
    orc_state_free(S);
    return rc;
}

/* ------------------------------------------------------------------------------------------- */
/* Operator-split scheme of the paper's Python tier (Sec. III B / III C), for comparison.        */
/* ------------------------------------------------------------------------------------------- */

/* Cavity slope at amplitude a and time t with the overlaps mm held fixed:
   (-i w - kappa) a + i g~ mm - i K |a|^2 a + eta(t). */
static void split_cavity_slope(const orc_problem *P, const double *a, const double *mm, double t,
                               double *da)
{
    for (int n = 0; n < P->nmodes; n++) {
        const double ar = a[2 * n], ai = a[2 * n + 1];
        const double gr = P->g_re[n], gi = P->g_im[n], mr = mm[2 * n], mi = mm[2 * n + 1];
        double r = -P->kappa[n] * ar + P->omega[n] * ai - (gr * mi + gi * mr);
        double i = -P->kappa[n] * ai - P->omega[n] * ar + (gr * mr - gi * mi);
        if (P->kerr) {
            const double k2 = P->kerr[n] * (ar * ar + ai * ai);
            r += k2 * ai;
            i -= k2 * ar;
        }
        da[2 * n] = r;
        da[2 * n + 1] = i;
    }
    if (P->drive_re) {
        const double x = (t - P->drive_t0) / P->drive_sigma;
        const double env = exp(-0.5 * x * x);
        for (int n = 0; n < P->nmodes; n++) {
            da[2 * n] += P->drive_re[n] * env;
            da[2 * n + 1] += P->drive_im[n] * env;
        }
    }
    add_pump(P, t, a, da);
}

/*
 * Lie splitting with interval ds, from S->t to T: at every interval start t_k = t_start + k ds
 * the cavity takes one classical RK4 step of length ds with the overlaps frozen at those of the
 * current magnetisation, then the magnet alone (cavity held at the new amplitudes, so the
 * feedback field is fixed) is integrated adaptively to t_{k+1}.  First order in ds.
 */
int orc_run_split(const orc_problem *P, orc_state *S, const orc_solver *sv, double T, double ds,
                  long max_attempts, orc_log *L)
{
    const int N = P->nmodes;
    if (!(ds > 0.0) || N > 64) return ORC_EINVAL;
    orc_problem Q = *P;
    Q.cavity_frozen = 1;
    double mm[128], k1[128], k2[128], k3[128], k4[128], y[128];
    const double t_start = S->t;
    for (long k = 0; S->t < T; k++) {
        double t1 = t_start + (double)(k + 1) * ds;
        if (t1 > T) t1 = T;
        const double h = t1 - S->t;
        orc_overlap(P, S->m, mm);
        split_cavity_slope(P, S->a, mm, S->t, k1);
        for (int q = 0; q < 2 * N; q++) y[q] = S->a[q] + 0.5 * h * k1[q];
        split_cavity_slope(P, y, mm, S->t + 0.5 * h, k2);
        for (int q = 0; q < 2 * N; q++) y[q] = S->a[q] + 0.5 * h * k2[q];
        split_cavity_slope(P, y, mm, S->t + 0.5 * h, k3);
        for (int q = 0; q < 2 * N; q++) y[q] = S->a[q] + h * k3[q];
        split_cavity_slope(P, y, mm, S->t + h, k4);
        for (int q = 0; q < 2 * N; q++)
            S->a[q] += h / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
        S->k1_valid = 0;   /* the feedback field changed with a */
        int rc = orc_run(&Q, S, sv, t1, max_attempts, L);
        if (rc) return rc;
        if (S->t < t1) return ORC_ESTEPFAIL;   /* attempt budget exhausted */
    }
    return ORC_OK;
}
