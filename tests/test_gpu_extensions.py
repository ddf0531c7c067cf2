"""Cavity-model extensions on the GPU (needs a B300): nonreciprocal coupling (backward
coefficient of the feedback field) and the self-Kerr term, against their closed form and the
FP64 oracle (1000 replayed steps, the adjoint's gradients)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

from gpu_util import TOL_A, TOL_M, f32_profiles, f32_state, replay_compare
from test_gpu_adjoint import TOL_G, compare, forward, loss_weights, oracle_grads, rel_err

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


def test_kerr_free_cavity_closed_form():
    a0 = 0.03 + 0.01j
    K = TP * 5e9
    p = W.make_problem(1, 1, 1, 10e-9, W.full_mask(1, 1, 1), B0=(0, 0, 0.2),
                       omega=[TP * 5.0e9], kappa=[TP * 30e6], g_re=[0.0], g_im=[0.0],
                       a0=np.array([a0]), rtol=1e-9, dt_max=2e-12,
                       m0=W.tilted_state(1, 1, 1, 1, 0.0, 0.0)).replace(kerr=np.array([K]))
    sim = cmx.Simulation.from_problem(p)
    T = 1.5e-9
    sim.run(T)
    a = sim.get_a()[0]
    sim.close()
    k, w = p.kappa[0], p.omega[0]
    th = np.angle(a0) - w * T - K * abs(a0) ** 2 * (1 - math.exp(-2 * k * T)) / (2 * k)
    want = abs(a0) * math.exp(-k * T) * np.exp(1j * th)
    assert abs(a - want) <= 1e-7 * abs(want), (a, want)


def extended_problem(T=1e-6, seed=4):
    n = 16
    p = W.make_problem(n, n, n, 10e-9, W.sphere_mask(n, n, n), alpha=1e-3,
                       B0=(0, 0, TP * 5e9 / W.GAMMA), Nd=(1 / 3, 1 / 3, 1 / 3),
                       omega=TP * np.array([5.0e9, 5.1e9]), kappa=TP * np.array([2e6, 4e6]),
                       g_re=TP * np.array([60e6, 30e6]), g_im=TP * np.array([0.0, 10e6]),
                       u=W.fourier_profiles(2, n, n, n, seed),
                       m0=W.tilted_state(1, n, n, n, 3.0, 0.2),
                       a0=np.array([0.01 + 0.002j, -0.004j]), T=T)
    p = p.replace(g_back=TP * np.array([25e6 + 5e6j, 70e6 - 10e6j]),
                  kerr=TP * np.array([4e10, -2e10]), dt_max=W.stable_dt_max(p))
    return f32_state(f32_profiles(p))


def test_nonreciprocal_kerr_replay_matches_oracle():
    dm, da, info = replay_compare(extended_problem(), 1000)
    assert dm <= TOL_M and da <= TOL_A, (dm, da)


def test_nonreciprocal_kerr_adjoint_matches_oracle():
    p = extended_problem(T=0.25e-9)
    sim, dts, traj = forward(p, 40)
    assert len(dts) > 80
    la, wm = loss_weights(p, traj)
    g = sim.adjoint(la, wm)
    sim.close()
    go = oracle_grads(p, dts, la, wm)
    errs = compare(p, g, go)
    for k in ("gb_re", "gb_im", "kerr"):
        errs[k] = rel_err(g[k], go[k])
    assert all(v <= TOL_G for v in errs.values()), errs
    # with separate backward coefficients the feedback gradients are not in g~'s
    assert np.abs(g["gb_re"]).max() > 0 and np.abs(g["kerr"]).max() > 0
