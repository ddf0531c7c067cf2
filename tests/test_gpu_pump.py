"""Degenerate parametric pump on the GPU (needs a B300): da_n/dt gains -i P_n e^{-i wp_n t}
conj(a_n) (the paper names parametric drives as a cavity-model swap in Sec. V; the reading is the
classical two-photon pump).  Checked against the free pumped cavity's closed form (below and
above threshold, complex pump, detuned), 1000 replayed steps of a coupled magnet + two pumped
modes against the FP64 oracle, the operator-split run against the oracle's, and the adjoint's
pump gradients against the oracle's adjoint."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

from gpu_util import TOL_A, TOL_M, f32_profiles, f32_state, masked, replay_compare
from test_gpu_adjoint import TOL_G, compare, forward, loss_weights, oracle_grads, rel_err
from test_oracle_pump import free_cavity_problem, pumped_cavity

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


@pytest.mark.parametrize("eps_over_kappa,phase,detune_MHz", [
    (0.5, 0.0, 0.0),      # below threshold
    (3.0, 0.0, 0.0),      # above threshold: one quadrature grows
    (2.0, 0.7, 0.0),      # complex pump
    (1.5, -1.1, 90.0),    # detuned beyond threshold: oscillating
])
def test_free_pumped_cavity_closed_form(eps_over_kappa, phase, detune_MHz):
    w, k = TP * 5.0e9, TP * 30e6
    P = eps_over_kappa * k * np.exp(1j * phase)
    wp = 2 * (w + TP * detune_MHz * 1e6)
    a0 = 0.03 + 0.01j
    p = free_cavity_problem(w, k, P, wp, a0, rtol=1e-9, dt_max=2e-12)
    T = 1.5e-9
    sim = cmx.Simulation.from_problem(p)
    st = sim.run(T)
    a = sim.get_a()[0]
    sim.close()
    assert abs(st["t"] - T) < 1e-21
    want = pumped_cavity(a0, w, k, P, wp, 0.0, T)
    # the cavity is FP64 on the device; the step control takes its error norm in FP32
    assert abs(a - want) <= 1e-7 * abs(want), (a, want)


def pumped_problem(T=1e-6, seed=5):
    n = 16
    p = W.make_problem(n, n, n, 10e-9, W.sphere_mask(n, n, n), alpha=1e-3,
                       B0=(0, 0, TP * 5e9 / W.GAMMA), Nd=(1 / 3, 1 / 3, 1 / 3),
                       omega=TP * np.array([5.0e9, 5.1e9]), kappa=TP * np.array([2e6, 4e6]),
                       g_re=TP * np.array([60e6, 30e6]), g_im=TP * np.array([0.0, 10e6]),
                       u=W.fourier_profiles(2, n, n, n, seed),
                       m0=W.tilted_state(1, n, n, n, 3.0, 0.2),
                       a0=np.array([0.01 + 0.002j, -0.004j]), T=T)
    p = p.replace(pump=TP * np.array([3e6 + 1e6j, -2e6 + 4e6j]),
                  pump_omega=TP * np.array([10.01e9, 10.2e9]), dt_max=W.stable_dt_max(p))
    return f32_state(f32_profiles(p))


def test_pumped_replay_matches_oracle():
    dm, da, info = replay_compare(pumped_problem(), 1000)
    assert dm <= TOL_M and da <= TOL_A, (dm, da)


def test_pumped_split_matches_the_oracle_split():
    p = f32_state(W.single_sphere().replace(dt_max=2e-13))
    w = p.omega[0]
    p = p.replace(pump=np.array([TP * 4e6 * np.exp(0.3j)]), pump_omega=np.array([2 * w]))
    T, ds = 0.5e-9, 2e-12
    sim = cmx.Simulation.from_problem(p, log_cap=0)
    sim.set_split(ds)
    st = sim.run(T)
    a, m = sim.get_a(), sim.get_m()
    sim.close()
    assert abs(st["t"] - T) < 1e-21
    it = O.Integrator(O.OracleProblem(p))
    rc, _ = it.run_split(T, ds)
    assert rc == 0
    o = it.state()
    m_o = o["m"].reshape(1, 3, p.nz, p.ny, p.nx)
    assert np.abs(a - o["a"]).max() <= 2e-3 * np.abs(o["a"]).max(), (a, o["a"])
    assert np.abs(masked(p, m) - masked(p, m_o)).max() <= 1e-4


def test_pumped_adjoint_matches_oracle():
    p = pumped_problem(T=0.25e-9)
    sim, dts, traj = forward(p, 40)
    assert len(dts) > 80
    la, wm = loss_weights(p, traj)
    g = sim.adjoint(la, wm)
    sim.close()
    go = oracle_grads(p, dts, la, wm)
    errs = compare(p, g, go)
    for k in ("pump_re", "pump_im"):
        errs[k] = rel_err(g[k], go[k])
    assert all(v <= TOL_G for v in errs.values()), errs
    assert np.abs(g["pump_re"]).max() > 0 and np.abs(g["pump_im"]).max() > 0


def test_pump_off_again():
    p = pumped_problem(T=0.05e-9)
    sim = cmx.Simulation.from_problem(p, log_cap=0)
    sim.set_pump(None)
    sim.run(p.T)
    a_off = sim.get_a()
    sim.close()
    q = p.replace(pump=None, pump_omega=None)
    sim = cmx.Simulation.from_problem(q, log_cap=0)
    sim.run(q.T)
    a_ref = sim.get_a()
    sim.close()
    assert np.array_equal(a_off, a_ref)
    with pytest.raises(cmx.CmxError):
        sim2 = cmx.Simulation.from_problem(q, log_cap=0)
        try:
            sim2.set_pump(np.array([np.nan, 0.0]), np.array([1.0, 1.0]))
        finally:
            sim2.close()
