"""External cavity drive on the GPU (needs a B300): the driven free cavity against its closed
form, replayed driven runs against the FP64 oracle (single problem, batch, adjoint)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

from gpu_util import TOL_A, TOL_M, f32_profiles, f32_state, masked, replay_compare
from test_oracle_drive import closed_form, free_cavity

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


def test_driven_free_cavity_matches_closed_form():
    p = free_cavity(drive=[3e7 + 1e7j, -2e7j], a0=(1e-3 + 2e-4j, 0), rtol=1e-9)
    p = p.replace(mask=np.ones((1, 1, 1), np.uint8), nx=1, ny=1, nz=1,
                  m0=W.tilted_state(1, 1, 1, 1, 0.0, 0.0))
    sim = cmx.Simulation.from_problem(p)
    for T in (0.05e-9, 0.12e-9, 0.5e-9):
        sim.run(T)
        a = sim.get_a()
        want = closed_form(p, T)
        assert np.abs(a - want).max() <= 2e-8 * np.abs(want).max(), (T, a, want)
    sim.close()


def driven_sphere(T=0.6e-9):
    """16^3 sphere, one cavity at the Kittel frequency pulsed at t0 = 0.1 ns (sigma = 20 ps)."""
    n = 16
    p = W.make_problem(n, n, n, 10e-9, W.sphere_mask(n, n, n), alpha=1e-3,
                       B0=(0, 0, TP * 5e9 / W.GAMMA), Nd=(1 / 3, 1 / 3, 1 / 3),
                       omega=[TP * 5e9, TP * 5.1e9], kappa=[TP * 2e6, TP * 4e6],
                       g_re=[TP * 50e6, TP * 30e6], g_im=[0.0, TP * 10e6],
                       u=W.fourier_profiles(2, n, n, n, 4),
                       m0=W.tilted_state(1, n, n, n, 0.0, 0.0), a0=np.zeros(2, complex), T=T)
    p = p.replace(drive=np.array([5e8, 2e8j]), dt_max=W.stable_dt_max(p))
    return f32_state(f32_profiles(p))


def test_driven_coupled_replay_matches_oracle():
    dm, da, info = replay_compare(driven_sphere(), 1000)
    assert info["stats"]["accepted"] >= 500
    assert np.abs(info["a_gpu"]).max() > 1e-4   # the pulse really excited the cavities
    assert dm <= TOL_M and da <= TOL_A, (dm, da)


def test_driven_adjoint_matches_oracle():
    from test_gpu_adjoint import compare, forward, oracle_grads, TOL_G
    p = driven_sphere(T=0.3e-9)
    sim, dts, traj = forward(p, 37)
    assert len(dts) > 2 * 37
    # a_0 = 0 here: energy in the last mode, unnormalised, plus random weights on all states
    rng = np.random.default_rng(3)
    la = rng.normal(size=(traj.shape[0], 2 * p.nmodes)) * 1e-2
    la[-1, -2:] += 2 * np.array([traj[-1, -1].real, traj[-1, -1].imag])
    wm = (rng.normal(size=(p.nsub, 3, p.nz, p.ny, p.nx)) * p.mask).astype(np.float32)
    g = sim.adjoint(la, wm)
    sim.close()
    errs = compare(p, g, oracle_grads(p, dts, la, wm))
    assert all(v <= TOL_G for v in errs.values()), errs


def test_driven_batch_matches_oracle():
    from test_gpu_batch import small_batch
    probs = [q.replace(drive=np.array([4e8, 1e8j, -2e8]), a0=np.zeros(q.nmodes, complex))
             for q in small_batch(n_inst=5, seed=9)]
    b = cmx.BatchSimulation(probs, log_cap=400)
    b.run(max_attempts=300)
    for i, p in enumerate(probs):
        log = b.get_log(i)
        dts = log["dt"][log["accepted"]]
        op = O.OracleProblem(p.replace(drive=p.drive[:p.nmodes]))
        it = O.Integrator(op)
        rc, olog = it.replay(dts)
        assert rc == 0
        st = it.state()
        m_orc = st["m"].reshape(1, 3, p.nz, p.ny, p.nx)
        assert np.abs(masked(p, b.get_m(i)) - masked(p, m_orc)).max() <= TOL_M
        amax = np.abs(olog.view()["a"]).max()
        assert amax > 1e-5
        assert np.abs(b.get_a(i) - st["a"]).max() <= TOL_A * amax
    b.close()


def pulsed_sweep(fm_list, T, g=TP * 50e6):
    """8^3 spheres, one cavity at 5 GHz pulsed at t0 = 0.1 ns, magnon frequency fm."""
    n = 8
    out = []
    for fm in fm_list:
        p = W.make_problem(n, n, n, 5e-9, W.sphere_mask(n, n, n), alpha=1e-4,
                           B0=(0, 0, TP * fm / W.GAMMA), Nd=(1 / 3, 1 / 3, 1 / 3),
                           omega=[TP * 5e9], kappa=[TP * 0.5e6], g_re=[g], g_im=[0.0],
                           m0=W.tilted_state(1, n, n, n, 0.0, 0.0), a0=np.zeros(1, complex),
                           T=T)
        out.append(p.replace(drive=np.array([2e8 + 0j])))
    return out


def hann_dft(t, y, f, t_start=0.0):
    keep = t >= t_start
    t, y = t[keep], y[keep]
    K = len(t)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(K) / (K - 1))
    return np.abs(np.exp(2j * np.pi * np.outer(f, t)) @ (w * y)) ** 2


def test_spectral_map_is_the_windowed_dft_of_the_trace():
    probs = pulsed_sweep([4.9e9, 5.0e9, 5.15e9], T=10e-9)
    b = cmx.BatchSimulation(probs, trace_cap=2000, sample_dt=10e-12)
    b.run()
    f = 4.7e9 + 2e6 * np.arange(300)
    P = b.spectrum(0, f[0], 2e6, len(f), t_start=0.2e-9)
    for i in range(len(probs)):
        tr = b.get_trace(i)
        want = hann_dft(tr["t"], tr["a"][:, 0], f, t_start=0.2e-9)
        assert np.abs(P[i] - want).max() <= 1e-9 * want.max(), i
    b.close()


def test_pulsed_field_sweep_spectral_peaks_follow_the_anticrossing():
    """The paper's spectroscopy (Sec. IV A): pulse the cavity, map the spectrum across the field
    sweep; the two strongest peaks sit on the branches of Eq. (6)."""
    from paper_2603_03706_b300 import spectra
    fms = [4.85e9, 4.95e9, 5.0e9, 5.05e9, 5.15e9]
    probs = pulsed_sweep(fms, T=100e-9)
    b = cmx.BatchSimulation(probs, trace_cap=6000, sample_dt=20e-12)
    b.run()
    df = 0.25e6
    f = 4.7e9 + df * np.arange(2400)
    P = b.spectrum(0, f[0], df, len(f), t_start=0.3e-9)
    b.close()
    for i, fm in enumerate(fms):
        s = P[i]
        peaks = [j for j in range(1, len(s) - 1) if s[j] >= s[j - 1] and s[j] > s[j + 1]]
        top = sorted(peaks, key=lambda j: -s[j])[:2]
        # parabolic refinement of each peak on the log power
        fp = []
        for j in top:
            l, c, r = np.log(s[j - 1]), np.log(s[j]), np.log(s[j + 1])
            fp.append(f[j] + 0.5 * df * (l - r) / (l - 2 * c + r))
        wp, wm = spectra.polariton_branches(TP * 5e9, TP * fm, TP * 50e6)
        want = sorted([wp.real / TP, wm.real / TP])
        assert np.abs(np.sort(fp) - want).max() <= 2e6, (fm, sorted(fp), want)
