"""Batched form: many instances in one persistent launch (needs a B300).

Each instance is checked against the FP64 oracle replaying its own accepted steps, against the
single-problem path replaying the same steps, for determinism, and a small field sweep across
the anticrossing against Eq. (6).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx, spectra
from paper_2603_03706_b300 import workloads as W

from gpu_util import TOL_A, TOL_M, check_step_log, f32_state, masked

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


def small_batch(n_inst=7, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n = int(rng.integers(6, 22))
        nm = int(rng.integers(1, 4))
        fm = 4.8e9 + 0.4e9 * i / max(n_inst - 1, 1)
        p = W.make_problem(n, n, n, 5e-9, W.sphere_mask(n, n, n), alpha=1e-3,
                           B0=(0, 0, TP * fm / W.GAMMA), Nd=(1 / 3, 1 / 3, 1 / 3),
                           omega=TP * rng.uniform(4.9e9, 5.1e9, nm),
                           kappa=TP * rng.uniform(1e6, 10e6, nm),
                           g_re=TP * rng.uniform(5e6, 80e6, nm), g_im=np.zeros(nm),
                           m0=W.tilted_state(1, n, n, n, 2.0, 0.3 * i),
                           a0=(rng.normal(size=nm) + 1j * rng.normal(size=nm)) * 1e-3, T=1e-6)
        out.append(f32_state(p))
    return out


@pytest.mark.parametrize("team", [1, 2])
def test_batch_instances_replay_against_oracle(team):
    probs = small_batch()
    b = cmx.BatchSimulation(probs, log_cap=600, team=team)
    b.run(max_attempts=500)
    for i, p in enumerate(probs):
        log = b.get_log(i)
        dts = log["dt"][log["accepted"]]
        assert len(dts) >= 400
        it = O.Integrator(O.OracleProblem(p))
        rc, olog = it.replay(dts)
        assert rc == 0
        st = it.state()
        m_orc = st["m"].reshape(1, 3, p.nz, p.ny, p.nx)
        dm = np.abs(masked(p, b.get_m(i)) - masked(p, m_orc)).max()
        da = np.abs(b.get_a(i) - st["a"]).max() / np.abs(olog.view()["a"]).max()
        assert dm <= TOL_M and da <= TOL_A, (i, dm, da)
        check_step_log(p, log, olog.view())
    b.close()


def medium_batch(sizes=(24, 30, 36, 42, 48), seed=17):
    """Spheres of 24^3 .. 48^3 cells (7,208 .. 57,864 magnetic cells), 1-3 modes each, B0 swept
    across the anticrossing: the lower end of the batched sweep's size range."""
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        nm = 1 + i % 3
        fm = 4.8e9 + 0.4e9 * i / max(len(sizes) - 1, 1)
        p = W.make_problem(n, n, n, 5e-9, W.sphere_mask(n, n, n), alpha=1e-3,
                           B0=(0, 0, TP * fm / W.GAMMA), Nd=(1 / 3, 1 / 3, 1 / 3),
                           omega=TP * np.array([5.0e9, 4.85e9, 5.15e9][:nm]),
                           kappa=TP * rng.uniform(1e6, 10e6, nm),
                           g_re=TP * rng.uniform(5e6, 80e6, nm), g_im=np.zeros(nm),
                           m0=W.tilted_state(1, n, n, n, 1.0, 0.7 * i),
                           a0=(rng.normal(size=nm) + 1j * rng.normal(size=nm)) * 1e-3, T=1e-6)
        out.append(f32_state(p))
    return out


@pytest.mark.parametrize("team", [8, 16])
def test_batch_medium_spheres_large_teams_replay_against_oracle(team):
    """Teams of 8 and 16 blocks (several segments per block, as in the benchmark's sweep) on
    24^3 .. 48^3 spheres: every instance's accepted steps replayed by the oracle, its error
    norms and step sizes checked attempt by attempt."""
    probs = medium_batch()
    b = cmx.BatchSimulation(probs, log_cap=420, team=team)
    assert b.info()["team_size"] == team
    b.run(max_attempts=400)
    for i, p in enumerate(probs):
        log = b.get_log(i)
        dts = log["dt"][log["accepted"]]
        assert len(dts) >= 300
        it = O.Integrator(O.OracleProblem(p))
        rc, olog = it.replay(dts)
        assert rc == 0
        st = it.state()
        m_orc = st["m"].reshape(1, 3, p.nz, p.ny, p.nx)
        dm = np.abs(masked(p, b.get_m(i)) - masked(p, m_orc)).max()
        da = np.abs(b.get_a(i) - st["a"]).max() / np.abs(olog.view()["a"]).max()
        assert dm <= TOL_M and da <= TOL_A, (i, dm, da)
        check_step_log(p, log, olog.view())
    b.close()


def test_batch_matches_single_problem_path():
    probs = small_batch(4, seed=9)
    b = cmx.BatchSimulation(probs, log_cap=300)
    b.run(max_attempts=200)
    for i, p in enumerate(probs):
        log = b.get_log(i)
        dts = log["dt"][log["accepted"]]
        sim = cmx.Simulation.from_problem(p)
        sim.replay(dts)
        assert np.abs(sim.get_m() - b.get_m(i)).max() < 1e-6
        assert np.abs(sim.get_a() - b.get_a(i)).max() < 1e-6 * max(np.abs(sim.get_a()).max(), 1e-12)
        sim.close()
    b.close()


def test_batch_deterministic():
    probs = small_batch(5, seed=3)
    res = []
    for _ in range(2):
        b = cmx.BatchSimulation(probs, log_cap=100)
        b.run(max_attempts=80)
        res.append([(b.get_m(i), b.get_a(i), b.get_log(i)["dt"]) for i in range(len(probs))])
        b.close()
    for r0, r1 in zip(*res):
        assert np.array_equal(r0[0], r1[0]) and np.array_equal(r0[1], r1[1])
        assert np.array_equal(r0[2], r1[2])


def test_batch_field_sweep_anticrossing_eq6():
    """Nine 8^3 spheres with B0 swept across the cavity resonance in one launch; the two branches
    of every instance follow Eq. (6)/(7) (Sec. IV A)."""
    wc, g = TP * 5e9, TP * 50e6
    probs = []
    for d in np.linspace(-120e6, 120e6, 9):
        p = W.single_sphere(T=20e-9)
        wm = wc + TP * d
        probs.append(p.replace(B0=np.array([0, 0, wm / W.GAMMA]),
                               m0=W.tilted_state(1, 8, 8, 8, 0.0, 0.0), a0=np.array([0.01 + 0j])))
    sdt = 5e-12
    b = cmx.BatchSimulation(probs, trace_cap=4200, sample_dt=sdt)
    b.run()
    for i, p in enumerate(probs):
        tr = b.get_trace(i)
        om, ga, amp = spectra.matrix_pencil(tr["a"][:, 0], sdt, 2)
        om = np.sort(om)
        wmL = W.GAMMA * p.B0[2] / (1 + p.alpha ** 2)
        bp, bm = spectra.polariton_branches(wc, wmL, g, p.kappa[0], p.alpha * wmL)
        assert np.abs(om - np.sort([bp.real, bm.real])).max() < TP * 0.5e6, i
    b.close()


def test_batch_rejects_profiles():
    p = W.multimode_sphere(nx=16, ny=16, nz=16)
    with pytest.raises(ValueError):
        cmx.BatchSimulation([p])


def test_batch_autotune_picks_a_runnable_shape():
    probs = small_batch(n_inst=9, seed=8)
    t = cmx.batch_autotune(probs, sample=5, attempts=4)
    assert (t["bx"], t["by"]) in ((32, 8), (32, 4)) and t["team"] >= 1, t
    assert len(t["us"]) == 12 and np.nanmin(t["us"]) > 0
    b = cmx.BatchSimulation(probs, log_cap=100, bx=t["bx"], by=t["by"], team=t["team"])
    st = b.run(max_attempts=50)
    assert st["attempts"] == 50 * len(probs) or st["t"] > 0
    for i, p in enumerate(probs):
        log = b.get_log(i)
        dts = log["dt"][log["accepted"]]
        it = O.Integrator(O.OracleProblem(p))
        rc, olog = it.replay(dts)
        assert rc == 0
        ost = it.state()
        m_orc = ost["m"].reshape(1, 3, p.nz, p.ny, p.nx)
        assert np.abs(masked(p, b.get_m(i)) - masked(p, m_orc)).max() <= TOL_M
    b.close()
