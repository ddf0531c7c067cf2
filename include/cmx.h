/*
 * cmx.h - C ABI of the device-resident cavity-magnonics integrator (sm_103a).
 *
 * The library advances the Landau-Lifshitz-Gilbert equation of a masked magnet coupled to N
 * cavity modes with an adaptive Dormand-Prince 5(4) scheme, entirely on the GPU.  Per stage it
 * evaluates (paper: "Multimode cavity magnonics in mumax+", arXiv 2603.03706):
 *   - the effective field: 6-neighbour exchange (free surface at the mask edge), uniaxial
 *     anisotropy, Zeeman, diagonal demag, inter-sublattice exchange for two sublattices
 *     (Sec. II G) and the cavity feedback B_rf,x(r) = sum_n u_n(r) (2/gamma) Re[g~_n a_n]
 *     (Eq. (3), (5), (13); complex g~ for dissipative coupling, Eq. (19));
 *   - the LLG torque with Gilbert damping (Sec. II A), Landau-Lifshitz form with 1/(1+alpha^2);
 *   - the overlaps <m^->_n = (1/N_c) sum_mask u_n (m_x - i m_y) (Eq. (2), (18));
 *   - the cavity ODEs da_n/dt = (-i w_n - kappa_n) a_n + i g~_n <m^->_n (Eq. (12), (19));
 *   - the stage combination, the max-norm error estimate and the accept/reject decision, so a
 *     run never returns to the host between steps (Sec. III A: one unified RK45 step with no
 *     host-side intervention).
 *
 * Conventions.  SI units; frequencies and rates in rad/s; fields in tesla.  Dense box arrays
 * are x fastest: index = x + nx*(y + ny*z).  Magnetisation arrays are [nsub][3][nx*ny*nz]
 * float32 (unit vectors; values outside the mask are ignored on input, written as 0 on
 * output).  Cavity amplitudes are interleaved complex float64: a[2n] = Re a_n, a[2n+1] = Im a_n.
 *
 * Memory.  The library copies every input at the call and owns all device memory it uses;
 * it never keeps a caller pointer.  "on_device" flags say whether a pointer is a device
 * address (read or written on the handle's stream) or host memory.
 *
 * Errors.  Every call returns a cmx_status.  Errors are sticky per handle: after a device-side
 * failure (NaN, step-size underflow, barrier time-out) later run calls return the same code
 * until cmx_set_state() resets the integrator.  cmx_last_error() gives a message owned by the
 * handle.  Handles are not thread-safe; use one host thread per handle.
 */
#ifndef CMX_H
#define CMX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CMX_OK = 0,
    CMX_EINVAL = 1,      /* bad argument (sizes, NULL pointers, unsupported combination) */
    CMX_ENOMEM = 2,      /* device or host allocation failed */
    CMX_ECUDA = 3,       /* a CUDA runtime call failed */
    CMX_ENAN = 4,        /* the error norm became NaN or Inf on the device */
    CMX_ESTEPFAIL = 5,   /* the step size fell below dt_min */
    CMX_ETIMEOUT = 6,    /* a device-side wait (grid barrier) exceeded its time limit */
    CMX_ESCRATCH = 7,    /* cmx_eval_rhs_noalloc: the problem does not fit the fixed scratch */
    CMX_ECHECK = 8       /* bounds-checked build (libcmx_check.so) only: a device index check
                            failed; the access was skipped and the run stopped (cmx_last_error
                            names the site and the index) */
} cmx_status;

#define CMX_MAX_MODES 8

typedef struct cmx_problem cmx_problem;   /* opaque handle */

/* Grid: nx*ny*nz cells of size cx*cy*cz metres; nsub = 1 (ferromagnet) or 2 (two-sublattice
 * antiferromagnet on the same cells).  nx <= 65535. */
typedef struct {
    int nx, ny, nz;
    double cx, cy, cz;
    int nsub;
} cmx_grid;

/* Material.  Ms [A/m] per sublattice, Aex [J/m] intra-sublattice exchange stiffness, alpha
 * Gilbert damping, gamma [rad/(s T)], Ku [J/m^3] along the unit vector ku_axis, B0 [T] static
 * field, Ndemag diagonal demag factors acting on the total moment Ms (m1 + m2), BE [T]
 * inter-sublattice exchange field (B_1 gets -BE m_2 and vice versa; ignored for nsub = 1). */
typedef struct {
    double Ms, Aex, alpha, gamma, Ku;
    double ku_axis[3];
    double B0[3];
    double Ndemag[3];
    double BE;
} cmx_material;

/* Cavity modes (n_modes <= CMX_MAX_MODES, may be 0).  omega, kappa, g_re, g_im: host arrays of
 * n_modes doubles; the complex coupling is g~_n = g_re[n] + i g_im[n] (g_d = -g_im, Eq. (19)).
 * u: n_modes x nx*ny*nz float32 mode profiles (dense box) or NULL for u_n = 1 everywhere;
 * u_on_device says where u lives. */
typedef struct {
    int n_modes;
    const double *omega, *kappa, *g_re, *g_im;
    const float *u;
    int u_on_device;
} cmx_modes;

/* Step-size control (the paper only says "adaptive RK45"; this is the reading used):
 *   err = max( max_cells |e_m| / rtol , max_n |e_a,n| / (rtol * max(a_ref, max_n |a_n|)) )
 *   accept iff err <= 1; dt <- min(dt * clamp(0.9 err^-1/5, 0.2, 5), dt_max), growth capped at
 *   1 right after a rejection; dt < dt_min -> CMX_ESTEPFAIL.
 * sample_dt > 0 records a uniform trace of a_n(t) (cubic Hermite) and <m^->_n(t) (linear) into
 * a device buffer of trace_cap samples.  log_cap: capacity of the per-attempt log. */
typedef struct {
    double rtol, a_ref, dt0, dt_min, dt_max;
    double sample_dt;
    int log_cap;
    int trace_cap;
} cmx_solver;

/* Launch shape.  A block of bx x by threads computes a tile of bx x by cells of a column of the
 * grid (one cell per thread, one warp per x-row) and loads the tile's one-cell rim as well; it
 * marches along z through its columns' planes.  Compiled tiles: 32x4, 32x8, 32x16, for one and
 * two sublattices; bx = by = 0 selects 32x8.  The columns' planes are split into contiguous
 * per-block segments with balanced plane counts; bz: the fewest planes per block (0 = 4); fewer
 * blocks are used when the grid is small.  blocks_per_sm caps the resident blocks per SM (0 =
 * as many as fit).  A grid magnetic over its whole box (a film, a full box: no mask) is stored
 * densely and its stages load each plane with tensor copies (cp.async.bulk.tensor, one thread
 * issuing a few per plane); plain_copies = 1 keeps the per-thread copies of masked grids for it
 * as well (0 = default; other values are rejected). */
typedef struct {
    int bx, by, bz;
    int blocks_per_sm;   /* 0 = as many as fit */
    int plain_copies;    /* 0 or 1 */
} cmx_tiling;

typedef struct {
    double t, dt;
    long long attempts, accepted;
    long long cell_stage_updates;   /* masked cells x RHS evaluations performed */
    int status;
    int launches;
} cmx_stats;

/* One per attempted step: end time (accepted) or start time (rejected), step size, scaled
 * error, accepted flag. */
typedef struct {
    double t, dt, err;
    int32_t accepted;
    int32_t pad;
} cmx_step;

/* Create a problem from the grid, the mask (host, nx*ny*nz bytes, nonzero = magnetic), the
 * material, the modes and the solver settings.  stream: a cudaStream_t (NULL = the legacy
 * default stream) on which all work of the handle is enqueued.  The initial state is m = +z
 * (sublattice 2: -z), a = 0, t = 0.  Fails with CMX_EINVAL for an empty mask, n_modes out of
 * range, nsub not 1 or 2, nx > 65535 or non-positive sizes. */
int cmx_create(const cmx_grid *grid, const uint8_t *mask, const cmx_material *mat,
               const cmx_modes *modes, const cmx_solver *solver, const cmx_tiling *tiling,
               void *stream, cmx_problem **out);

int cmx_destroy(cmx_problem *h);

/* Set y = (m, a) at time t and reset the step size to dt0 (m: dense box [nsub][3][nbox]
 * float32, host or device; a: 2*n_modes doubles on the host, may be NULL = zeros). */
int cmx_set_state(cmx_problem *h, const float *m, int m_on_device, const double *a, double t);

/* Adaptive integration until t >= T (the final attempt is shortened to land on T) or until
 * max_attempts attempts have been made (<= 0: no limit).  Blocks the calling thread; the work
 * runs as persistent kernel launches on the handle's stream, each ending after at most
 * cmx_set_launch_attempts() attempts, with one small status read between launches. */
int cmx_run(cmx_problem *h, double T, long long max_attempts, cmx_stats *st);

/* Enqueue ONE launch of up to n_attempts adaptive attempts towards T; does not wait. */
int cmx_launch(cmx_problem *h, double T, int n_attempts);

/* Replay: take exactly the n given step sizes (host array), every step accepted. */
int cmx_replay(cmx_problem *h, const double *dts, long long n, cmx_stats *st);

/* Wait for the handle's stream and return the integrator status and counters. */
int cmx_sync(cmx_problem *h, cmx_stats *st);

/* Evaluate the right-hand side once at (m, a) without touching the integrator state:
 * dm (dense box, same layout as m, 0 outside the mask), da (2N), mm (2N: <m^->_n).  All host
 * pointers.  Uses the same stage kernel as the integrator (stage 1). */
int cmx_eval_rhs(cmx_problem *h, const float *m, const double *a, float *dm, double *da,
                 double *mm);

/* Results.  m: dense box [nsub][3][nbox] float32 (host or device).  a: 2N doubles (host). */
int cmx_get_m(cmx_problem *h, float *dst, int on_device);
int cmx_get_a(cmx_problem *h, double *dst);

/* Per-attempt log (cap entries; *n receives the number of attempts logged so far, which may
 * exceed the log capacity).  a, mm: optional (cap * 2N doubles): amplitudes after each accepted
 * attempt and the overlap <m^->_n at its 5th-order point. */
int cmx_get_log(cmx_problem *h, cmx_step *dst, double *a, double *mm, int cap, long long *n);

/* Uniform trace: t (cap), a (cap*2N), mm (cap*2N), host pointers; *n = samples recorded. */
int cmx_get_trace(cmx_problem *h, double *t, double *a, double *mm, int cap, long long *n);

/* Number of magnetic cells and number of stored cells (stored = magnetic + padding holes). */
int cmx_ncells(const cmx_problem *h, long long *n_magnetic, long long *n_stored);

/* Attempts per persistent launch in cmx_run (default 4096). */
int cmx_set_launch_attempts(cmx_problem *h, int n);

/* Device-side wait limit for grid barriers in nanoseconds (default 2e9). */
int cmx_set_timeout(cmx_problem *h, long long ns);

/* Test hook: block `block` of the next launch skips its first barrier arrival and exits, so
 * the other blocks reach their wait limit; -1 disables.  Used only to test CMX_ETIMEOUT. */
int cmx_debug_skip_arrival(cmx_problem *h, int block);

/* External drive of the cavities (Eq. (1), (12)): eta_n(t) = (eta_re + i eta_im)_n
 * exp(-(t - t0)^2 / (2 sigma^2)) is added to da_n/dt, evaluated at each stage's time (the
 * Gaussian pulse of Sec. IV A: sigma = 20 ps, t0 = 0.1 ns).  eta_re, eta_im: host, n_modes
 * each [1/s]; eta_re == NULL switches the drive off.  Applies to the following launches. */
int cmx_set_drive(cmx_problem *h, const double *eta_re, const double *eta_im, double t0,
                  double sigma);

/* Operator-split scheme of the paper's Python tier (Sec. III B/C), for comparison with the coupled
 * integrator: every interval ds the cavity takes one classical RK4 step with the overlaps held at
 * those of the current magnetisation, then the magnet alone is integrated adaptively to the next
 * boundary with the cavity (and so the feedback field) held fixed.  First order in ds; still one
 * persistent launch (the boundaries and cavity steps are handled by the device controller).
 * ds = 0 returns to the coupled scheme.  Applies from the current state on; replays and the
 * adjoint use the coupled scheme (cmx_adjoint_record fails while it is on). */
int cmx_set_split(cmx_problem *h, double ds);

/* Nonreciprocal coupling (Sec. II: separate forward and backward coefficients, h0 = 2 g_b /
 * gamma): the feedback field uses B_rf,x = sum_n u_n (2/gamma) Re[gb~_n a_n] with the backward
 * coefficients gb~ given here (host, n_modes each), while the cavity equation keeps the forward
 * g~ of cmx_modes.  gb_re == NULL restores reciprocal coupling. */
int cmx_set_backward_coupling(cmx_problem *h, const double *gb_re, const double *gb_im);

/* Self-Kerr cavity term -i K_n |a_n|^2 a_n [rad/s per |a|^2] (host, n_modes; NULL: none). */
int cmx_set_kerr(cmx_problem *h, const double *kerr);

/* Degenerate parametric pump (Sec. V lists parametric drives as a cavity-model swap without a
 * formula; this is the classical equation of a two-photon pump): da_n/dt gains
 * -i P_n e^{-i wp_n t} conj(a_n), P_n = p_re[n] + i p_im[n] [rad/s], pump frequency wp[n]
 * [rad/s], phase referenced to t = 0, evaluated at each stage's time t + c_s h.  Host arrays of
 * n_modes; p_re == NULL removes the pump.  Above threshold (|P|^2 > kappa^2 + (wp/2 - w)^2)
 * the cavity grows exponentially, as the equation says.  The operator-split scheme takes it in
 * its cavity step; the adjoint returns dL/d Re P_n and dL/d Im P_n (cmx_grads.pump_re/pump_im).
 * CMX_EINVAL for a non-finite coefficient. */
int cmx_set_pump(cmx_problem *h, const double *p_re, const double *p_im, const double *wp);

/* Autotuner: time `attempts` Dormand-Prince attempts (after a one-attempt warm-up) from the
 * current state with each compiled tile (32x4, 32x8, 32x16; blocks_per_sm and bz of the
 * current tiling) and, for a grid small enough, with the single-block integrator, restore the
 * state after each trial (m, FSAL slope, control block; the step log and trace counters roll
 * back too) and keep the fastest.  *chosen (may be NULL) receives it (bx = by = 0: the
 * single-block integrator); us_per_attempt (may be NULL, 4 entries) the measured times in that
 * order (NaN where a candidate does not apply; with full demag only 32x8 is timed). */
int cmx_autotune(cmx_problem *h, int attempts, cmx_tiling *chosen, double *us_per_attempt);

/* Full magnetostatic demag (mode 1) instead of the diagonal factors Ndemag of cmx_material
 * (mode 0, the default).  The field of the magnetic cells is the convolution
 * B_d(r_i) = -mu0 Ms sum_j N(r_i - r_j) m_j with the cell-pair tensor of Newell, Williams and
 * Dunlop (1993), evaluated on the device in every stage by zero-padded FFTs; for two
 * sublattices it acts on the total moment m1 + m2.  The paper notes that diagonal factors hold
 * only for the uniform mode of an ellipsoid (Sec. II C, Eq. (9)); the full field is what
 * non-uniform modes (Sec. II D, Eq. (11)) and non-ellipsoidal samples need.  Grids up to
 * CMX_DEMAG_MAX_FFT / 2 cells per axis.  With mode 1 the single-block integrator is not used,
 * and the adjoint (cmx_adjoint_record) is rejected; the batched form has no full demag.
 * Returns CMX_EINVAL for a larger grid, a recording adjoint or another mode. */
#define CMX_DEMAG_MAX_FFT 256
int cmx_set_demag(cmx_problem *h, int mode);

/* Checkpoint and resume (no counterpart in the paper): cmx_save_state writes into the host
 * buffer `blob` (cap bytes) the integrator's state: the control block (time, step size, cavity
 * amplitudes and slopes, counters, step-log and trace positions, controller flags) and the
 * stored state m_n and FSAL slope of every cell; *size (may be NULL) receives the byte count
 * (blob == NULL: size query only).  cmx_load_state puts such a blob into a handle created for
 * the same grid, mask, sublattices and mode count (CMX_EINVAL otherwise) and configured the same
 * way (solver, drive, couplings, split, demag: those are not in the blob); a run continued from
 * it is bitwise the run continued from the saved handle.  The step log and trace buffers keep
 * their contents; new entries continue at the saved positions.  A replay in progress is not
 * resumed, and loading ends any checkpoint recording for the adjoint.  Both synchronise. */
int cmx_save_state(cmx_problem *h, void *blob, size_t cap, size_t *size);
int cmx_load_state(cmx_problem *h, const void *blob, size_t size);

/* Planning query, host only (no device work, callable without a GPU): the row-compacted layout
 * and the partition that `blocks` blocks of bx x by tiles would use for this grid and mask
 * (mask: host, nx*ny*nz, x fastest).  *n_segments (may be NULL) receives the number of column
 * segments, *n_stored (may be NULL) the number of stored cells (rows padded to 8 cells).
 * Returns CMX_EINVAL if the tile is not compiled, the mask is empty, or the tile columns cannot
 * be spread over `blocks` blocks of at most 64 segments each (cmx_create and cmx_batch_create
 * reject such a problem with the same code instead of leaving cells out). */
int cmx_plan_tiling(const cmx_grid *grid, const uint8_t *mask, int bx, int by, int blocks,
                    long long *n_segments, long long *n_stored);

/* Launch shape actually used: bx, by, bz, grid blocks, segments; *dense = 1 when the stages
 * take the tensor-copy path of dense boxes (0: per-thread copies, or the single-block
 * integrator).  Every pointer may be NULL. */
int cmx_get_tiling(const cmx_problem *h, int *bx, int *by, int *bz, int *blocks, int *tiles,
                   int *dense);

const char *cmx_last_error(const cmx_problem *h);

/* 1 for the bounds-checked build of this library (libcmx_check.so: every stage kernel checks
 * its shared- and global-memory indices, CMX_ECHECK on a failed check), 0 for libcmx.so. */
int cmx_checked_build(void);
const char *cmx_status_string(int status);

/* ------------------------------------------------------------------------------------------
 * Right-hand-side evaluation without device allocation (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc: plug-ins living inside a host program whose own
 * allocator owns all device memory (a cudaMalloc behind its back breaks its accounting or
 * fails because it has reserved the memory), and services under a fixed device-memory budget
 * that must not meet an out-of-memory error after start-up.  It computes the same f(m, a) as
 * cmx_eval_rhs, with the
 * same stage kernel, but allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * routine.  Every scratch buffer (compact layout tables, compact m and slope, control block,
 * block partials) is carved from one file-scope device array of CMX_NOALLOC_SCRATCH_BYTES
 * (16 MiB), which every GPU that loads the library holds until the process exits.
 *
 * grid, mask (host), mat, modes (u host or device, or NULL): as for cmx_create.
 * m: DEVICE pointer, dense box [nsub][3][nbox] float32 (read on `stream`).
 * a: host, 2N doubles (NULL = zeros).  dm: DEVICE pointer, dense box like m, written with the
 * slopes (0 outside the mask).  da, mm: host, 2N doubles each (may be NULL).
 * stream: cudaStream_t (NULL = legacy default stream); the call waits for it before returning.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture starts.  All calls share
 * the one array and it keeps the last call's contents: calls that overlap on the GPU (other
 * host threads, other streams) race and must be serialised by the caller.
 * Returns CMX_ESCRATCH when the problem's buffers need more than CMX_NOALLOC_SCRATCH_BYTES
 * (28 bytes per stored cell for one sublattice with no profiles, about 600k cells; with two
 * host-side profiles 44 bytes, about 380k cells), CMX_EINVAL on bad arguments. */
#define CMX_NOALLOC_SCRATCH_BYTES (16u << 20)
int cmx_eval_rhs_noalloc(const cmx_grid *grid, const uint8_t *mask, const cmx_material *mat,
                         const cmx_modes *modes, const float *m, const double *a, float *dm,
                         double *da, double *mm, void *stream);

/* ------------------------------------------------------------------------------------------
 * Batched form: many independent problems (e.g. a field sweep across the anticrossing, Sec.
 * IV A, or a cooperativity sweep, Sec. IV C) advanced by ONE persistent launch.  Each instance
 * has its own grid, mask, material, modes, end time, adaptive step size, controller, log and
 * trace.  The launch's blocks form teams of equal size; each team integrates the instances of
 * its queue one after the other (longest first, queues balanced by cell count), with a barrier
 * counter of its own instead of a grid-wide barrier.  All instances must share nsub and use
 * uniform mode profiles (modes.u = NULL).
 * ---------------------------------------------------------------------------------------- */
typedef struct cmx_batch cmx_batch;

/* One instance: grid, host mask, material, modes (u must be NULL), optional host initial state
 * (m0: dense box [nsub][3][nbox] float32, NULL = +z / -z; a0: 2N doubles, NULL = 0) and the
 * end time T of its integration. */
typedef struct {
    cmx_grid grid;
    const uint8_t *mask;
    cmx_material mat;
    cmx_modes modes;
    const float *m0;
    const double *a0;
    double T;
} cmx_instance;

/* bx, by: block window (as cmx_tiling; 0 = 32x8).  team: blocks per team (0 = smallest power of
 * two for which the largest instance fits the average team load).  blocks_per_sm: cap (0 = as
 * many as fit).  use_graph: capture each launch in a CUDA graph and replay it (1) or launch
 * directly (0). */
typedef struct {
    int bx, by;
    int team;
    int blocks_per_sm;
    int use_graph;
} cmx_batch_config;

/* Create a batch of n instances sharing the solver settings (log_cap / trace_cap apply per
 * instance).  Copies everything; owns all device memory.  CMX_EINVAL on an empty mask, mixed
 * nsub, non-NULL profiles, n <= 0. */
int cmx_batch_create(const cmx_instance *inst, int n, const cmx_solver *solver,
                     const cmx_batch_config *cfg, void *stream, cmx_batch **out);
int cmx_batch_destroy(cmx_batch *b);

/* Batch autotuner: for every candidate launch shape (tile 32x8 or 32x4, times team size
 * automatic, 1, 2, 4, 8, 16), build a trial batch over every k-th
 * instance (k = ceil(n / sample)), time one launch of `attempts` attempts per instance with CUDA
 * events after a one-attempt warm-up launch, and destroy it.  cfg is read for use_graph and
 * blocks_per_sm and receives the fastest bx, by, team.  us (may be NULL, 12 entries) gets the
 * time of each candidate in microseconds (NaN: not runnable), *ncand the number of candidates. */
int cmx_batch_autotune(const cmx_instance *inst, int n, const cmx_solver *solver, int sample,
                       int attempts, void *stream, cmx_batch_config *cfg, double *us,
                       int *ncand);

/* The same drive for every instance: n_eta amplitudes (host arrays, n_eta <= CMX_MAX_MODES) for
 * modes 0 .. n_eta-1, zero for higher modes; instance i uses its first n_modes(i).  See
 * cmx_set_drive; eta_re == NULL switches the drive off. */
int cmx_batch_set_drive(cmx_batch *b, const double *eta_re, const double *eta_im, int n_eta,
                        double t0, double sigma);

/* Spectral map of the field sweep (the paper's spectra, Sec. IV A): for every instance,
 * P_i(f) = |sum_k w_k a_mode(t_k) e^{+2 pi i f t_k}|^2 over its uniform trace samples with
 * t_k >= t_start (Hann window w over those samples; the trace needs trace_cap > 0 and
 * sample_dt > 0), at f = f0 + j df, j < nf [Hz].  out: host, n x nf doubles (row of an
 * instance without mode `mode`: zeros).  Computed on the device from the device-resident
 * traces. */
int cmx_batch_spectrum(cmx_batch *b, int mode, double f0, double df, int nf, double t_start,
                       double *out);

/* Enqueue ONE launch in which every unfinished instance makes up to n_attempts attempts. */
int cmx_batch_launch(cmx_batch *b, int n_attempts);

/* Launch until every instance has reached its T (or failed), at most max_attempts attempts per
 * instance (<= 0: no limit); *total sums the counters over instances (t = smallest t).  Returns
 * the first instance error, if any. */
int cmx_batch_run(cmx_batch *b, long long max_attempts, cmx_stats *total);

/* Per-instance results (host pointers), same layouts as the single-problem calls. */
int cmx_batch_stats(cmx_batch *b, int i, cmx_stats *st);
int cmx_batch_get_a(cmx_batch *b, int i, double *a);
int cmx_batch_get_m(cmx_batch *b, int i, float *m);
int cmx_batch_get_log(cmx_batch *b, int i, cmx_step *dst, double *a, double *mm, int cap,
                      long long *n);
int cmx_batch_get_trace(cmx_batch *b, int i, double *t, double *a, double *mm, int cap,
                        long long *n);

/* Launch shape: teams, blocks per team, total blocks, total magnetic cells, graph in use. */
int cmx_batch_info(const cmx_batch *b, int *teams, int *team_size, int *blocks,
                   long long *cells, int *graph);
const char *cmx_batch_last_error(const cmx_batch *b);

/* ---------------------------------------------------------------------------------------------
 * Adjoint form: gradients through the accepted steps of a run
 *
 * The paper integrates forward only; this is the differentiation form built beside it.  For a
 * loss L(a_0, a_1, ..., a_n, m_n) of the cavity amplitudes after every accepted step (a_0: the
 * initial amplitudes) and the final magnetisation, cmx_adjoint returns dL/d(Re g~_n),
 * dL/d(Im g~_n), dL/d kappa_n, dL/d omega_n, dL/d alpha, dL/d u_n(r) and dL/d(a_0, m_0): the
 * discrete adjoint of exactly the computation the run performed (its stages, the FSAL slope of
 * the un-normalised 5th-order point, the renormalisation of m on accept), with the accepted
 * step sizes held fixed (a step-size change is not differentiated).
 *
 *   cmx_set_state(h, m0, ..., a0, t0);
 *   cmx_adjoint_record(h, every, max_steps);  // arm the checkpoint store (allocates)
 *   cmx_run(h, T, 0, &st);                    // forward; checkpoints every `every` accepted steps
 *   cmx_adjoint(h, dL_da, dL_dm, 0, &grads);  // reverse sweep
 *
 * Memory: checkpoints hold 2 x nsub*3 FP32 per stored cell plus 6N doubles per slot
 * (max_steps/every + 1 slots); the reverse sweep recomputes one checkpoint interval at a time and
 * keeps its stage points (every x 6 x nsub*3 FP32 per stored cell) plus twelve per-cell arrays.
 * ------------------------------------------------------------------------------------------- */

/* Gradients written by cmx_adjoint.  Every pointer may be NULL (that gradient is skipped). */
typedef struct {
    double *g_re, *g_im;   /* host, n_modes each: dL/d Re g~_n, dL/d Im g~_n (rad/s)^-1 */
    double *kappa, *omega; /* host, n_modes each */
    double *alpha;         /* host, 1 */
    double *a0;            /* host, 2N packed (Re, Im): dL/d a_0 */
    float *m0;             /* dense nsub*3*nbox: dL/d m_0 of the normalised initial state; 0
                              outside the mask */
    int m0_on_device;      /* m0 is a device pointer */
    double *u;             /* dense N*nbox: dL/d u_n(r); needs mode profiles; 0 outside */
    int u_on_device;       /* u is a device pointer */
    double *gb_re, *gb_im; /* host, n_modes each: dL/d of the backward coupling (zero unless set
                              by cmx_set_backward_coupling; otherwise in g_re, g_im) */
    double *kerr;          /* host, n_modes: dL/d K_n */
    double *pump_re, *pump_im; /* host, n_modes each: dL/d Re P_n, dL/d Im P_n of the pump */
} cmx_grads;

/* Arm the checkpoint store for the next run: call after cmx_set_state and before any launch.
 * every >= 1 accepted steps between checkpoints; max_steps bounds the accepted steps the run
 * may take (a run that takes more makes cmx_adjoint fail with CMX_EINVAL).  cmx_set_state
 * disarms it.  The run's step log must hold all of its attempts (solver.log_cap). */
int cmx_adjoint_record(cmx_problem *h, int every, long long max_steps);

/* Reverse sweep over the accepted steps of the run since cmx_adjoint_record.
 * dL_da: host, (n+1) x 2N doubles, row i = dL/d a_i packed (Re, Im), n = accepted steps (the
 *        a_i are the step log's amplitudes of the accepted attempts, a_0 the initial ones);
 *        NULL = zero.
 * dL_dm: dense nsub*3*nbox FP32, dL/d m_n (host, or device if dL_dm_on_device); NULL = zero.
 * Writes the gradients requested in g.  The handle's own state (m, a, t) is not changed; the run
 * may be differentiated again with another loss.  Errors: CMX_EINVAL if nothing was recorded,
 * if the run took more than max_steps accepted steps or the step log overflowed; device errors
 * as cmx_run (CMX_ETIMEOUT, CMX_ENAN). */
int cmx_adjoint(cmx_problem *h, const double *dL_da, const float *dL_dm, int dL_dm_on_device,
                cmx_grads *g);

/* Accepted steps recorded since cmx_adjoint_record (n of the loss above). */
int cmx_adjoint_steps(cmx_problem *h, long long *n);

#ifdef __cplusplus
}
#endif
#endif /* CMX_H */
