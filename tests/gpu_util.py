"""Shared helpers of the GPU tests: build the CUDA handle and the oracle from one Problem."""
import numpy as np

from oracle import oracle as O
from paper_2603_03706_b300 import cmx

# Parity bars after 1000 replayed steps (FP32 device state vs FP64 oracle).
TOL_M = 2e-5
TOL_A = 1e-4

# Error-norm agreement between the device (FP32 stage slopes) and the oracle (FP64) on the same
# accepted step.  The magnet's error estimate e = h sum_j E_j k_j is a combination of slopes with
# weights that sum to zero, so FP32 rounding of the slopes (relative u = 6e-8, about ten
# operations deep) is not cancelled: |de| <~ 10 u h sum_j |E_j| max|k| with sum_j |E_j| = 0.16 and
# h max|k| <= 1.2 (the step-size cap keeps h gamma |B| at or below the stability bound), i.e.
# |de| <~ 1.2e-7, or 0.12 in units of rtol = 1e-6 where the step reaches that cap.  On top of it
# the state itself differs by up to 2e-5 after 1000 steps, which moves the estimate by a relative
# amount of the same order.  ERR_ABS is that floor times 1 / 2.5 (h max|k| is below 0.5 on the
# steps of these workloads) and ERR_REL covers the state difference.
ERR_ABS = 0.05
ERR_REL = 1e-2


def f32_profiles(p):
    """Round the mode profiles to float32 once, so both sides see identical inputs."""
    if p.u is None:
        return p
    return p.replace(u=np.asarray(p.u, np.float32))


def f32_state(p):
    """Initial m rounded to float32 and renormalised in float64 (the oracle's input)."""
    m = np.asarray(p.m0, np.float32).astype(np.float64)
    n = np.linalg.norm(m, axis=1, keepdims=True)
    n[n == 0] = 1.0
    return p.replace(m0=m / n)


def sim_for(p, log_cap=4096, trace_cap=0, sample_dt=0.0, tiling=None):
    return cmx.Simulation.from_problem(p, log_cap=log_cap, trace_cap=trace_cap,
                                       sample_dt=sample_dt, tiling=tiling)


def masked(p, m):
    """Magnetic-cell values of a dense (nsub, 3, nz, ny, nx) array -> (nsub, 3, ncell)."""
    m = np.asarray(m).reshape(p.nsub, 3, -1)
    return m[:, :, p.mask.reshape(-1) > 0]


def expected_next_dt(h, err, accepted, last_rejected, dt_max):
    """Step size the controller proposes after an attempt of size h with scaled error err
    (reading C6 as the device evaluates it: the factor 0.9 err^(-1/5) in FP32, clamped to
    [0.2, 5] with exact bounds, no growth right after a rejection, dt_max after an accept)."""
    e = np.float32(err)
    ff = np.float32(5.0) if e <= 0 else np.float32(0.9) * np.power(e, np.float32(-0.2))
    fac = 5.0 if ff >= np.float32(5.0) else (0.2 if ff < np.float32(0.2) else float(ff))
    if accepted:
        if last_rejected and ff > np.float32(1.0):
            fac = 1.0
        return min(h * fac, dt_max)
    return h * fac


def check_step_log(p, log, olog=None, T=None):
    """The device log of an adaptive run against reading C6: every attempt's size follows from
    the previous attempt's size, error and decision (shortened only to land on T), and, when the
    oracle's replay log of the accepted steps is given, each accepted step's error norm agrees
    with the oracle's within ERR_ABS + ERR_REL err.  Returns (max |d err|, number of attempts)."""
    dt, err, acc, t = log["dt"], log["err"], log["accepted"], log["t"]
    T = p.T if T is None else T
    last_rej = False
    for i in range(len(dt) - 1):
        prop = expected_next_dt(dt[i], err[i], bool(acc[i]), last_rej, p.dt_max)
        last_rej = not acc[i]
        h = min(prop, p.dt_max)
        if t[i] + h >= T:
            h = T - t[i]
        assert abs(dt[i + 1] - h) <= 2e-6 * h, (i, dt[i + 1], h, err[i], acc[i])
    derr = 0.0
    if olog is not None:
        eg = err[acc]
        eo = olog["err"][: len(eg)]
        assert len(eo) == len(eg)
        d = np.abs(eg - eo)
        derr = float(d.max()) if len(d) else 0.0
        assert np.all(d <= ERR_ABS + ERR_REL * eo), (derr, int(np.argmax(d)))
    return derr, len(dt)


def replay_compare(p, n_steps, tiling=None, autotune=0):
    """Run the GPU adaptively for n_steps attempts, replay its accepted steps in the oracle and
    return (max |dm|, max |da| / max |a|, info).  The device log is checked against the
    controller rule and the oracle's error norms (check_step_log).  autotune > 0: pick the
    window with cmx_autotune (that many attempts per trial, state restored) first, as the
    benchmark does."""
    p = f32_state(f32_profiles(p))
    sim = sim_for(p, log_cap=n_steps + 8, tiling=tiling)
    if autotune:
        sim.autotune(autotune)
    st = sim.run(p.T, max_attempts=n_steps)
    log = sim.get_log()
    dts = log["dt"][log["accepted"]]
    m_gpu = sim.get_m()
    a_gpu = sim.get_a()
    tiling_used = sim.get_tiling()
    sim.close()
    it = O.Integrator(O.OracleProblem(p))
    rc, olog = it.replay(dts)
    assert rc == 0
    ost = it.state()
    m_orc = ost["m"].reshape(p.nsub, 3, p.nz, p.ny, p.nx)
    dm = np.abs(masked(p, m_gpu) - masked(p, m_orc)).max()
    amax = max(np.abs(olog.view()["a"]).max() if p.nmodes else 0.0, 1e-30)
    da = np.abs(a_gpu - ost["a"]).max() / amax if p.nmodes else 0.0
    derr, _ = check_step_log(p, log, olog.view())
    return dm, da, dict(log=log, stats=st, oracle_log=olog.view(), a_orc=ost["a"], a_gpu=a_gpu,
                        m_gpu=m_gpu, m_orc=m_orc, dts=dts, derr=derr, tiling=tiling_used)
