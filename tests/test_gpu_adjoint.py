"""Adjoint form on the GPU (needs a B300): the CUDA reverse sweep against the FP64 oracle's
discrete adjoint on the same recorded step sequence, against central finite differences of the
CUDA forward itself, and its invariances (checkpoint spacing, determinism).

The loss touches every state the adjoint returns: a weighted sum of all cavity amplitudes
a_0 .. a_n, the energy transferred into one mode, and a weighted final magnetisation.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

from gpu_util import f32_profiles, f32_state, masked

pytestmark = pytest.mark.gpu
TP = 2 * math.pi

# Gradient parity bar (FP32 reverse sweep vs FP64 oracle, per gradient kind, relative to the
# largest entry of that kind): the stage points and slope adjoints are FP32 like the forward,
# the scalar chain FP64.
TOL_G = 2e-3


def sphere16(T=0.3e-9):
    """16^3 copy of the adjoint workload (sphere, three profiled modes, a_1(0) = 0.01)."""
    return f32_state(f32_profiles(W.adjoint_sphere(T=T, n=16)))


def afm_small(T=0.05e-9):
    nx, ny, nz = 24, 20, 4
    mask = W.random_mask(nx, ny, nz, 0.9, 3)
    p = W.make_problem(nx, ny, nz, 2e-9, mask, nsub=2, Ms=4e5, Aex=5e-12, alpha=2e-3, Ku=5e4,
                       B0=(0, 0, 1.0), Nd=(0, 0, 1), BE=50.0, omega=TP * np.array([150e9]),
                       kappa=TP * np.array([50e6]), g_re=TP * np.array([2e9]),
                       g_im=TP * np.array([0.2e9]),
                       u=W.fourier_profiles(1, nx, ny, nz, 5), T=T,
                       m0=W.random_state(2, nx, ny, nz, 4, spread=0.1, afm=True),
                       a0=np.array([0.01 + 0.003j]))
    p = p.replace(dt_max=W.stable_dt_max(p))
    return f32_state(f32_profiles(p))


def ferro_plain(T=0.2e-9):
    """No mode profiles (u = 1), holes in the mask, complex coupling."""
    nx, ny, nz = 29, 13, 9
    mask = W.random_mask(nx, ny, nz, 0.85, 8)
    p = W.make_problem(nx, ny, nz, 5e-9, mask, Ku=-610.0, ku_axis=(0.6, 0.0, 0.8),
                       B0=(0.01, 0, 0.187), Nd=(0.3, 0.3, 0.4), alpha=0.01,
                       omega=TP * np.array([5.0e9, 5.2e9]), kappa=TP * np.array([2e6, 4e6]),
                       g_re=TP * np.array([60e6, 30e6]), g_im=TP * np.array([-10e6, 20e6]),
                       m0=W.random_state(1, nx, ny, nz, 9, spread=0.2),
                       a0=np.array([0.004 - 0.002j, 0.003j]), T=T)
    return f32_state(p.replace(dt_max=W.stable_dt_max(p)))


def forward(p, every, max_steps=100000, tiling=None):
    sim = cmx.Simulation.from_problem(p, log_cap=max_steps + 64, tiling=tiling)
    sim.adjoint_record(every, max_steps)
    st = sim.run(p.T)
    log = sim.get_log()
    acc = log["accepted"]
    traj = np.concatenate([np.asarray(p.a0, complex)[None], log["a"][acc]]) if p.nmodes else None
    return sim, log["dt"][acc], traj


def loss_weights(p, traj, seed=0, target=None):
    """dL/da (packed reals, (n+1) x 2N) and dL/dm for the test loss."""
    rng = np.random.default_rng(seed)
    n1, N = traj.shape
    la = rng.normal(size=(n1, 2 * N)) * 1e-2
    i, j = (0, N - 1) if target is None else target
    e0 = abs(traj[0, i]) ** 2
    la[-1, 2 * j] += 2 * traj[-1, j].real / e0
    la[-1, 2 * j + 1] += 2 * traj[-1, j].imag / e0
    wm = rng.normal(size=(p.nsub, 3, p.nz, p.ny, p.nx)) * p.mask
    return la, wm.astype(np.float32)


def oracle_grads(p, dts, la, wm):
    op = O.OracleProblem(p)
    return O.adjoint(op, op.m0(), O.pack_a(p.a0), dts, la,
                     np.asarray(wm, np.float64).reshape(-1))


def rel_err(x, ref):
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


def compare(p, g, go):
    errs = dict(g_re=rel_err(g["g_re"], go["g_re"]), g_im=rel_err(g["g_im"], go["g_im"]),
                kappa=rel_err(g["kappa"], go["kappa"]), omega=rel_err(g["omega"], go["omega"]),
                alpha=rel_err(g["alpha"], go["alpha"]), a0=rel_err(g["a0_packed"], go["a0"]))
    m_o = go["m0"].reshape(p.nsub, 3, p.nz, p.ny, p.nx)
    errs["m0"] = rel_err(masked(p, g["m0"]), masked(p, m_o))
    if p.u is not None:
        u_o = go["u"].reshape(p.nmodes, -1)[:, p.mask.reshape(-1) > 0]
        u_g = g["u"].reshape(p.nmodes, -1)[:, p.mask.reshape(-1) > 0]
        errs["u"] = rel_err(u_g, u_o)
    return errs


@pytest.mark.parametrize("case,every,tiling", [("sphere16", 40, None), ("afm", 16, None),
                                               ("plain", 25, None),
                                               ("sphere16", 40, (32, 4, 1))])
def test_adjoint_matches_oracle(case, every, tiling):
    p = {"sphere16": sphere16, "afm": afm_small, "plain": ferro_plain}[case]()
    sim, dts, traj = forward(p, every, tiling=tiling)
    assert len(dts) > 2 * every, len(dts)   # several intervals and a partial last one
    la, wm = loss_weights(p, traj)
    g = sim.adjoint(la, wm)
    sim.close()
    assert g["n"] == len(dts)
    go = oracle_grads(p, dts, la, wm)
    errs = compare(p, g, go)
    bad = {k: v for k, v in errs.items() if not v <= TOL_G}
    assert not bad, errs


def test_checkpoint_spacing_does_not_change_the_gradient():
    p = sphere16(T=0.12e-9)
    res = []
    for every in (1, 13, 100000):
        sim, dts, traj = forward(p, every)
        la, wm = loss_weights(p, traj)
        res.append(sim.adjoint(la, wm))
        sim.close()
    for g in res[1:]:
        for k in ("g_re", "g_im", "kappa", "omega", "a0_packed"):
            assert np.allclose(g[k], res[0][k], rtol=1e-10, atol=0), k
        assert abs(g["alpha"] - res[0]["alpha"]) <= 1e-10 * abs(res[0]["alpha"])
        assert np.array_equal(g["m0"], res[0]["m0"])
        assert rel_err(g["u"], res[0]["u"]) <= 1e-5


def test_adjoint_is_deterministic_and_repeatable():
    p = sphere16(T=0.1e-9)
    sim, dts, traj = forward(p, 20)
    la, wm = loss_weights(p, traj)
    g1 = sim.adjoint(la, wm)
    g2 = sim.adjoint(la, wm)   # the same recorded run, differentiated again
    a_after = sim.get_a()
    sim.close()
    for k in ("g_re", "g_im", "kappa", "omega", "a0_packed", "m0", "u"):
        assert np.array_equal(g1[k], g2[k]), k
    assert g1["alpha"] == g2["alpha"]
    assert np.allclose(a_after, traj[-1], rtol=0, atol=0)   # the run's own state is untouched


def replay_loss(p, dts, j):
    """Energy transferred into mode j, |a_j(T)|^2 / |a_1(0)|^2, of a replay of dts."""
    sim = cmx.Simulation.from_problem(p, log_cap=0)
    sim.replay(dts)
    a = sim.get_a()
    sim.close()
    return abs(a[j]) ** 2 / abs(p.a0[0]) ** 2


def test_energy_transfer_gradient_matches_central_differences():
    """Central differences of the CUDA forward on the frozen step sequence (h = 1e-4
    relative).  FP32 rounding of the two replays limits agreement to about 1e-3 here."""
    p = sphere16(T=2e-9)
    sim, dts, traj = forward(p, 200)
    N = p.nmodes
    la = np.zeros((len(dts) + 1, 2 * N))
    e0 = abs(p.a0[0]) ** 2
    la[-1, 2 * (N - 1)] = 2 * traj[-1, N - 1].real / e0
    la[-1, 2 * (N - 1) + 1] = 2 * traj[-1, N - 1].imag / e0
    g = sim.adjoint(la, None)
    sim.close()
    L0 = abs(traj[-1, N - 1]) ** 2 / e0
    assert L0 > 1e-6
    checks = [("g_re", 0), ("g_re", 2), ("kappa", 0), ("kappa", 2), ("g_im", 0), ("g_im", 2),
              ("omega", 0), ("omega", 2), ("g_re", 1)]
    checked = 0
    for name, n in checks:
        v = np.array(getattr(p, name), float)
        step = max(abs(v[n]), TP * 1e6)
        # FD resolves only parameters the loss is sensitive to: FP32 rounding of L is about
        # 1e-6 L, i.e. 1e-6 L / (2 h) in the difference quotient
        if abs(g[name][n]) * step < 1e-2 * L0:
            continue
        h = 1e-4 * step
        vp, vm = v.copy(), v.copy()
        vp[n] += h
        vm[n] -= h
        fd = (replay_loss(p.replace(**{name: vp}), dts, N - 1) -
              replay_loss(p.replace(**{name: vm}), dts, N - 1)) / (2 * h)
        assert abs(fd - g[name][n]) <= 2e-2 * abs(g[name][n]) + 1e-6 * L0 / (2 * h), \
            (name, n, fd, g[name][n])
        checked += 1
    assert checked >= 4, checked


def test_adjoint_errors():
    p = sphere16(T=0.02e-9)
    sim = cmx.Simulation.from_problem(p, log_cap=64)
    with pytest.raises(cmx.CmxError):
        sim.adjoint(None, None)            # nothing recorded
    sim.run(0.01e-9)
    with pytest.raises(cmx.CmxError):
        sim.adjoint_record(10, 1000)       # not right after set_state
    sim.set_state(p.m0, p.a0)
    sim.adjoint_record(5, 3)               # at most 3 accepted steps
    sim.run(p.T)
    with pytest.raises(cmx.CmxError):
        sim.adjoint(None, None)
    sim.close()


def test_autograd_function_matches_the_direct_call():
    """torch.autograd through CoupledRun gives the gradients of cmx_adjoint for the same loss."""
    import torch
    from paper_2603_03706_b300 import adjoint as AD
    p = sphere16(T=0.2e-9)
    prm = AD.parameters_from(p)
    spec = AD.RunSpec(problem=p, every=50, max_steps=20000)
    a_traj, t, m_T = AD.run(prm["g_re"], prm["g_im"], prm["kappa"], prm["omega"], prm["alpha"],
                            prm["u"], prm["a0"], prm["m0"], spec)
    L = AD.energy_transfer(a_traj, 0, 2)
    L.backward()
    # the same loss through the C call
    sim, dts, traj = forward(p, 50)
    N = p.nmodes
    la = np.zeros((len(dts) + 1, 2 * N))
    e0 = abs(traj[0, 0]) ** 2
    eT = abs(traj[-1, 2]) ** 2
    la[-1, 4:6] = 2 * np.array([traj[-1, 2].real, traj[-1, 2].imag]) / e0
    la[0, 0:2] = -2 * eT / e0 ** 2 * np.array([traj[0, 0].real, traj[0, 0].imag])
    g = sim.adjoint(la, None)
    sim.close()
    assert abs(float(L) - eT / e0) <= 1e-12 * eT / e0
    for k in ("g_re", "g_im", "kappa", "omega"):
        # entries far below the largest one come from cancellations: compare on its scale
        ref = np.abs(g[k]).max()
        assert np.allclose(prm[k].grad.numpy(), g[k], rtol=1e-12, atol=1e-12 * ref), k
    assert abs(float(prm["alpha"].grad) - g["alpha"]) <= 1e-12 * abs(g["alpha"])
    # dL/da_0 sums the direct term of |a_1(0)|^2 and the adjoint's: compare on its scale
    ga = np.stack([g["a0"].real, g["a0"].imag], -1)
    assert np.allclose(prm["a0"].grad.numpy(), ga, rtol=0, atol=1e-12 * np.abs(ga).max())
    assert np.allclose(prm["u"].grad.numpy(), g["u"].astype(np.float32), rtol=1e-6, atol=0)


def two_mode_resonant(T=5e-9):
    """16^3 sphere, one cavity at the Kittel frequency, g/2pi = 50 MHz: two polariton branches
    about 100 MHz apart (Eq. (7))."""
    n = 16
    B0 = TP * 5e9 / W.GAMMA
    p = W.make_problem(n, n, n, 10e-9, W.sphere_mask(n, n, n), alpha=1e-4, B0=(0, 0, B0),
                       Nd=(1 / 3, 1 / 3, 1 / 3), omega=[TP * 5e9], kappa=[TP * 0.5e6],
                       g_re=[TP * 50e6], g_im=[0.0], m0=W.tilted_state(1, n, n, n, 0.0, 0.0),
                       a0=np.array([0.01 + 0j]), T=T)
    return f32_state(p.replace(dt_max=W.stable_dt_max(p)))


def test_splitting_gradient_matches_central_differences():
    import torch
    from paper_2603_03706_b300 import adjoint as AD
    p = two_mode_resonant()
    prm = AD.parameters_from(p)
    spec = AD.RunSpec(problem=p, every=200, max_steps=40000)
    a_traj, t, _ = AD.run(prm["g_re"], prm["g_im"], prm["kappa"], prm["omega"], prm["alpha"],
                          None, prm["a0"], prm["m0"], spec)
    S = AD.splitting(a_traj, t, 0)
    S.backward()
    # the branches of Eq. (7) at resonance are 2 g apart
    assert abs(float(S) - 2 * p.g_re[0]) <= 0.05 * 2 * p.g_re[0]
    # frozen steps, central differences of the CUDA forward and the same estimator
    sim, dts, _ = forward(p, 200)
    sim.close()

    def S_of(gre):
        sm = cmx.Simulation.from_problem(p.replace(g_re=np.array([gre])), log_cap=len(dts) + 8)
        sm.replay(dts)
        lg = sm.get_log()
        sm.close()
        tr = np.concatenate([p.a0[None], lg["a"]])
        at = torch.tensor(np.stack([tr.real, tr.imag], -1))
        tt = torch.tensor(np.concatenate([[0.0], lg["t"]]))
        return float(AD.splitting(at, tt, 0))

    h = 1e-3 * p.g_re[0]
    fd = (S_of(p.g_re[0] + h) - S_of(p.g_re[0] - h)) / (2 * h)
    ad = float(prm["g_re"].grad[0])
    assert abs(fd - ad) <= 2e-2 * abs(fd), (fd, ad)
    assert 1.5 < ad < 2.5   # dS/dg close to 2 at resonance
