"""The paper's closed forms reproduced by the CUDA integrator (needs a B300).

Spectral peaks of the device trace are located with the matrix-pencil estimator and compared
with Eq. (6)/(7) (anticrossing, Sec. II B), Eq. (9) (Kittel), Eq. (20) (level attraction) and
with the FP64 oracle's trace of the same problem (within 1 MHz); the dark state of Eq. (14),
the vacuum Rabi period pi/g (Sec. IV B) and the overlap selection rule (Eq. (10)-(11)) are
checked directly.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx, spectra
from paper_2603_03706_b300 import workloads as W

pytestmark = pytest.mark.gpu
TP = 2 * math.pi
SDT = 5e-12


def gpu_trace(p, T, sample_dt=SDT):
    n = int(T / sample_dt) + 2
    sim = cmx.Simulation.from_problem(p, trace_cap=n, sample_dt=sample_dt)
    st = sim.run(T)
    tr = sim.get_trace()
    sim.close()
    assert st["status"] == 0
    return tr


def oracle_trace(p, T, sample_dt=SDT):
    """Oracle on a fixed grid of sample_dt steps (replay), amplitudes at every sample."""
    n = int(round(T / sample_dt))
    it = O.Integrator(O.OracleProblem(p))
    rc, log = it.replay(np.full(n, sample_dt))
    assert rc == 0
    v = log.view()
    a = np.concatenate([O.unpack_a(O.OracleProblem(p).a0())[None, :], v["a"]])
    return np.concatenate([[0.0], v["t"]]), a


def branches(y, order=2):
    om, ga, amp = spectra.matrix_pencil(y, SDT, order)
    o = np.argsort(om[:order])
    return om[:order][o], ga[:order][o]


def resonant_sphere(B0=None, g=TP * 50e6, a0=0.01):
    p = W.single_sphere()
    if B0 is not None:
        p = p.replace(B0=np.array([0, 0, B0]))
    return p.replace(g_re=np.array([g]), m0=W.tilted_state(1, 8, 8, 8, 0.0, 0.0),
                     a0=np.array([a0 + 0j]))


@pytest.mark.parametrize("detune_MHz", [0.0, -40.0, 60.0])
def test_anticrossing_branches_match_eq6_and_oracle(detune_MHz):
    wc = TP * 5e9
    wm = wc + TP * detune_MHz * 1e6
    p = resonant_sphere(B0=wm / W.GAMMA * (1 + 1e-6))
    T = 20e-9
    tr = gpu_trace(p, T)
    om, ga = branches(tr["a"][:, 0])
    wmL = W.GAMMA * p.B0[2] / (1 + p.alpha ** 2)
    gm = p.alpha * wmL
    bp, bm = spectra.polariton_branches(wc, wmL, p.g_re[0], p.kappa[0], gm)
    want = np.sort([bp.real, bm.real])
    assert np.abs(om - want).max() < TP * 0.5e6, (om / TP, want / TP)
    # the oracle's trace of the same problem gives the same branches within 1 MHz
    t, a = oracle_trace(p, T)
    om_o, _ = branches(a[:, 0])
    assert np.abs(om - om_o).max() < TP * 1e6


def test_kittel_frequency_uncoupled():
    p = W.single_sphere().replace(g_re=np.array([0.0]))
    tr = gpu_trace(p, 10e-9)
    om, ga = spectra.matrix_pencil(tr["mm"][:, 0], SDT, 1)[:2]
    w = W.GAMMA * p.B0[2] / (1 + p.alpha ** 2)
    assert abs(om[0] - w) < TP * 0.5e6
    assert abs(ga[0] - p.alpha * w) < TP * 0.2e6


def test_vacuum_rabi_period_pi_over_g():
    g = TP * 100e6
    p = resonant_sphere(g=g)
    tr = gpu_trace(p, 16e-9, sample_dt=2e-12)
    a2 = np.abs(tr["a"][:, 0]) ** 2
    t = tr["t"]
    idx = [i for i in range(1, len(a2) - 1) if a2[i] < a2[i - 1] and a2[i] <= a2[i + 1]
           and a2[i] < 0.2 * a2.max()]
    tm = []
    for i in idx:
        A = np.polyfit(t[i - 1:i + 2], a2[i - 1:i + 2], 2)
        tm.append(-A[1] / (2 * A[0]))
    periods = np.diff(tm)
    assert len(periods) >= 2
    assert np.abs(periods / (math.pi / g) - 1).max() < 3e-3


def test_dark_mode_stays_dark():
    g1, g2, w, k = TP * 40e6, TP * 70e6, TP * 5e9, TP * 3e6
    eps = 1e-2 / math.hypot(g1, g2)
    p = W.make_problem(8, 8, 8, 5e-9, W.sphere_mask(8, 8, 8), B0=(0, 0, w / W.GAMMA),
                       Nd=(1 / 3, 1 / 3, 1 / 3), omega=[w, w], kappa=[k, k], g_re=[g1, g2],
                       g_im=[0, 0], m0=W.tilted_state(1, 8, 8, 8, 0.0, 0.0),
                       a0=np.array([eps * g2, -eps * g1], complex), rtol=1e-8)
    T = 2e-9
    sim = cmx.Simulation.from_problem(p)
    sim.run(T)
    m = sim.get_m().reshape(3, -1)[:, p.mask.reshape(-1) > 0]
    a = sim.get_a()
    sim.close()
    assert np.abs(m[:2]).max() < 1e-6
    want = np.array([eps * g2, -eps * g1]) * np.exp(-(1j * w + k) * T)
    assert np.abs(a - want).max() < 1e-5 * np.abs(want).max()


def test_level_attraction_eq20():
    gd = TP * 50e6
    p = resonant_sphere(g=0.0, a0=1e-3).replace(g_im=np.array([-gd]))
    tr = gpu_trace(p, 8e-9)
    om, ga = branches(tr["a"][:, 0])
    wc = p.omega[0]
    wmL = W.GAMMA * p.B0[2] / (1 + p.alpha ** 2)
    bp, bm = spectra.polariton_branches(wc, wmL, -1j * gd, p.kappa[0], p.alpha * wmL)
    # real parts coalesce, imaginary parts split by about 2 g_d
    assert abs(om[0] - om[1]) < TP * 2e6
    assert abs(abs(ga[0] - ga[1]) - abs(bp.imag - bm.imag)) < TP * 1e6


def test_overlap_selection_rule_on_device():
    n = 16
    u = W.cos_profiles([0, 1, 2, 3], n, n, n)
    p = W.make_problem(n, n, n, 5e-9, W.sphere_mask(n, n, n), omega=[TP * 5e9] * 4,
                       kappa=[0] * 4, g_re=[0] * 4, g_im=[0] * 4, u=u)
    m = W.tilted_state(1, n, n, n, 20.0, 0.7)
    sim = cmx.Simulation.from_problem(p)
    _, _, mm = sim.eval_rhs(np.asarray(m, np.float32), np.zeros(4, complex))
    sim.close()
    mminus = math.sin(math.radians(20)) * np.exp(-0.7j)
    assert abs(mm[0] - mminus) < 1e-6
    assert abs(mm[1]) < 1e-6 and abs(mm[3]) < 1e-6
