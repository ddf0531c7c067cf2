"""Shared helpers of the GPU tests: build the CUDA handle and the oracle from one Problem."""
import numpy as np

from oracle import oracle as O
from paper_2603_03706_b300 import cmx

# Parity bars after 1000 replayed steps (FP32 device state vs FP64 oracle).
TOL_M = 2e-5
TOL_A = 1e-4


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


def replay_compare(p, n_steps, tiling=None):
    """Run the GPU adaptively for n_steps attempts, replay its accepted steps in the oracle and
    return (max |dm|, max |da| / max |a|, gpu log)."""
    p = f32_state(f32_profiles(p))
    sim = sim_for(p, log_cap=n_steps + 8, tiling=tiling)
    st = sim.run(p.T, max_attempts=n_steps)
    log = sim.get_log()
    dts = log["dt"][log["accepted"]]
    m_gpu = sim.get_m()
    a_gpu = sim.get_a()
    sim.close()
    it = O.Integrator(O.OracleProblem(p))
    rc, olog = it.replay(dts)
    assert rc == 0
    ost = it.state()
    m_orc = ost["m"].reshape(p.nsub, 3, p.nz, p.ny, p.nx)
    dm = np.abs(masked(p, m_gpu) - masked(p, m_orc)).max()
    amax = max(np.abs(olog.view()["a"]).max() if p.nmodes else 0.0, 1e-30)
    da = np.abs(a_gpu - ost["a"]).max() / amax if p.nmodes else 0.0
    return dm, da, dict(log=log, stats=st, oracle_log=olog.view(), a_orc=ost["a"], a_gpu=a_gpu,
                        m_gpu=m_gpu, m_orc=m_orc, dts=dts)
