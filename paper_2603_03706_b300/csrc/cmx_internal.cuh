// Internal definitions shared by the sm_103a kernels and the host code of libcmx.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cmx.h"

// CMX_CHECK = 1 builds the bounds-checked library: the stage kernels verify their shared- and
// global-memory indices; a failed check skips the access and stops the run with CMX_ECHECK.
#ifndef CMX_CHECK
#define CMX_CHECK 0
#endif

namespace cmx {

constexpr int MAXN = CMX_MAX_MODES;

// Mode constants held per mode by the device code: w, kappa, Re g~, Im g~ (forward coupling, in
// the cavity equation), Re gb~, Im gb~ (backward coupling, in the feedback field) and the
// self-Kerr coefficient K.
constexpr int MC = 7;

// Row storage alignment in cells: every row's stored span starts at a multiple of ROW_ALIGN
// cells of x and of the compact index (see cmx_layout.h), so that a tile row (x0 a multiple of
// 32) starts on a 32-byte sector.
constexpr int ROW_ALIGN = 8;

// Longest segment (planes including its two halo planes) and most segments per block.
constexpr int MAX_TILE_PLANES = 66;
constexpr int MAX_BLOCK_SEGMENTS = 64;

// Dormand & Prince (1980) 5(4) coefficients, written from the published rationals.
// dp_a(s, j): coupling of stage s+1 to slope j+1 (row 6 is the 5th-order solution, FSAL).
// dp_e(j) = b5_j - b4_j (5th minus embedded 4th-order weight) for the error estimate.
// Both are constexpr so that, with the stage index a template parameter, zero couplings are
// removed at compile time (stage 7 never reads slope 2).
__host__ __device__ constexpr double dp_a(int s, int j)
{
    constexpr double A[7][6] = {
        {0, 0, 0, 0, 0, 0},
        {1.0 / 5, 0, 0, 0, 0, 0},
        {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
        {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
        {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
        {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
        {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84},
    };
    return A[s][j];
}

// Node c_s of stage s+1: the row sum of its couplings (the stage's time is t + c_s h).
__host__ __device__ constexpr double dp_c(int s)
{
    return dp_a(s, 0) + dp_a(s, 1) + dp_a(s, 2) + dp_a(s, 3) + dp_a(s, 4) + dp_a(s, 5);
}

// Doubles per checkpoint slot of the adjoint store: a, k1^a, <m^-> (2N each) and the time.
__host__ __device__ constexpr int traj_stride(int nmodes)
{
    return 6 * nmodes + 2;
}

__host__ __device__ constexpr double dp_e(int j)
{
    constexpr double E[7] = {71.0 / 57600, 0, -71.0 / 16695, 71.0 / 1920,
                             -17253.0 / 339200, 22.0 / 525, -1.0 / 40};
    return E[j];
}

// Fixed-point scale of the overlap sums: the largest power of two (at most 2^40) that keeps a
// sum of magnitude up to `bound` (max |u| times the magnetic cells) below 2^61.
inline double overlap_scale(double bound)
{
    int e = 61 - (int)std::ceil(std::log2(bound > 1.0 ? bound : 1.0));
    if (e > 40) e = 40;
    return std::ldexp(1.0, e);
}

// Integrator control block in device memory.  Written only by the block that completes a
// grid barrier (the "controller"), read by every block after the barrier is released.
struct Ctl {
    double t, dt, T;                 // current time, proposed step, end time of this run
    double a[2 * MAXN];              // cavity amplitudes at t
    double ka[7][2 * MAXN];          // cavity slopes of the current attempt (logical order)
    double mm_n[2 * MAXN];           // overlap <m^->_n at t (for trace interpolation)
    int kphys[7];                    // physical k buffer of logical slope j
    int mcur;                        // m buffer holding y_n
    int k1_valid;                    // FSAL slope of y_n present
    int last_rejected;
    int status;                      // sticky cmx_status
    int done;                        // stop this launch
    int replay;                      // 1: take step sizes from replay_dts
    long long attempts, accepted, launch_attempts, max_launch_attempts;
    long long rhs_evals;             // RHS evaluations (stages) performed
    long long replay_pos, replay_n;
    const double *replay_dts;
    long long log_n, trace_n;
    double trace_next;
    // operator-split scheme (Ctx::split_dt > 0): next interval boundary, its index, the grid's
    // origin, and a cavity step still to be taken at the current boundary
    double split_next, split_t0;
    long long split_k;
    int split_pending;
    unsigned int bar_count, bar_gen; // grid barrier
    // Grid sums of the stage's overlaps as fixed-point integers (value x red_scale), and the bit
    // pattern of the grid max of |e_m|, in three sets used in turn by stage count mod 3: the
    // blocks add into the current set before the barrier; the set for two stages ahead is
    // cleared by the team's rank 0 after it.  Integer addition makes the sum independent of the
    // order of arrival.
    long long racc[3][2 * MAXN];
    unsigned int remax[3];
    int range_error;                 // a block partial left the fixed-point range
    int skip_block;                  // test hook (see cmx_debug_skip_arrival)
    int timeout_where;               // barrier or index-check site of the stopping error
    long long check_value;           // bounds-checked build: the offending index
};

// Kernel arguments (by value).
struct Ctx {
    int nx, ny, nz, nsub, nmodes;
    int ncell;                       // stored cells (compact, incl. padding holes)
    int ncell_mag;                   // magnetic cells N_c
    const int2 *rows;                // per (z, y) row: x = offset, y = xs | xe << 16
    const uint32_t *active;          // bitmask over stored cells (NULL: no holes)
    const int4 *tiles;               // segments: x0, y0, z0, z1
    const int *seg_begin;            // block b owns segments [seg_begin[b], seg_begin[b+1])
    int ntiles, bz;
    int nxs;                         // stored row length of a dense box (nx rounded up to 8)
    int dense;                       // 1: every row is magnetic over the whole box and the
                                     // launch takes the dense tensor-copy stage path
    const float *u;                  // [nmodes][ncell] or NULL
    float *m[2];                     // [nsub*3][ncell]
    float *k[7];                     // [nsub*3][ncell]
    // stored stage values: stage S (2..6) writes m_{S+1} into msv[(S+1) & 1], stage S+1 reads
    // its tile and halo from there; es: the error partial sum_{j<=6} E_j k_j of stage 6
    float *msv[2];                   // [nsub*3][ncell]
    float *es;                       // [nsub*3][ncell]
    // full magnetostatic demag (fd = 1; dmg is then 0): tensor spectrum [6][Lz][Ly][Lx] (real,
    // scaled), FFT work array [3][nz][Ly][Lx], the field of the stage value bd [3][ncell] and
    // the twiddles of the three axes (see cmx_demag.cuh)
    int fd;
    const float *dk;
    float2 *dwork;
    float *bd;
    const float2 *dtw[3];
    int Lx, Ly, Lz, lgx, lgy, lgz;
    // material (float, tesla units)
    float wx, wy, wz;                // (2 Aex / Ms) / c_d^2
    float anis, ku[3], B0[3], dmg[3], BE;
    float pre, alpha;                // -gamma/(1+alpha^2), alpha
    // modes
    double omega[MAXN], kappa[MAXN], gre[MAXN], gim[MAXN];
    double gbre[MAXN], gbim[MAXN];   // backward (feedback) coupling; equal to g~ unless set
    double kerr[MAXN];               // self-Kerr -i K |a|^2 a (0: none)
    // degenerate parametric pump -i P_n e^{-i wp_n t} conj(a_n) on da_n/dt, P_n = pump_re +
    // i pump_im [rad/s] at pump frequency pump_w [rad/s]; has_pump = 0: none
    double pump_re[MAXN], pump_im[MAXN], pump_w[MAXN];
    int has_pump;
    int has_gb;                      // 1: nonreciprocal coupling (gradients of gb~ separate)
    double two_over_gamma, inv_nmag;
    double red_scale;                // fixed-point scale of the overlap sums (a power of two)
    float umax;                      // bound on |u_n(r)| (1 without profiles)
    // external drive eta_n(t) = drive_n exp(-(t - drive_t0)^2 / (2 sigma^2)) on da_n/dt
    // (Eq. (1), (12)); has_drive = 0: none
    double drive_re[MAXN], drive_im[MAXN];
    double drive_t0, drive_inv_sigma;
    int has_drive;
    // solver
    double rtol, a_ref, dt_min, dt_max, sample_dt;
    Ctl *ctl;
    // log / trace
    cmx_step *log;
    double *log_a, *log_mm;
    int log_cap;
    double *tr_t, *tr_a, *tr_mm;
    int tr_cap;
    long long timeout_ns;
    int stage_only;                  // 1: evaluate stage 1 once (cmx_eval_rhs) and stop
    double split_dt;                 // > 0: operator-split scheme with this interval
    // Checkpoint store of the adjoint (NULL = off): slot k holds the state after
    // k * traj_every accepted steps counted from traj_base (slot 0: the initial state):
    // m (renormalised) and the FSAL slope k1, and a, k1^a and <m^-> at the slope's point.
    float *traj_m, *traj_k;          // [slot][nsub*3][ncell]
    double *traj_a;                  // [slot][traj_stride(N)]: a, k1^a, <m^->, t
    long long traj_base;
    int traj_every, traj_slots;
    // Stage record of a replay (NULL = off): replay step j stores its stage points
    // m_S (S = 2..7) and, for every stage it evaluates, a_S and <m^->_S.
    float *rec_m;                    // [j][S-2][nsub*3][ncell]
    double *rec_a;                   // [j][S-1][2][2N]
    double *rec_t;                   // [j]: start time of replay step j
    int rec_steps;
};

}  // namespace cmx
