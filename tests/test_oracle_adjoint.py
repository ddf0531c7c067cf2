"""Pins of the oracle's discrete adjoint (CPU only).

The adjoint is tied to things other than itself: central finite differences of the oracle's own
forward map (the right-hand side, then whole replayed step sequences, for every parameter kind),
and a closed form (a free cavity decays as exp(-kappa t), so d|a(T)|^2/d kappa = -2 T |a(T)|^2).
A dropped term, a wrong sign or a transposed operand in any transposed piece moves one of these
by far more than the tolerance.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import workloads as W

TP = 2 * math.pi


def ferro_case(seed=1):
    """Small ferromagnet with holes, two profiled modes, complex coupling, tilted anisotropy."""
    nx, ny, nz = 6, 5, 4
    mask = W.random_mask(nx, ny, nz, 0.8, seed)
    u = W.fourier_profiles(2, nx, ny, nz, seed + 7).astype(np.float64)
    ku = np.array([0.3, -0.2, 1.0])
    ku /= np.linalg.norm(ku)
    p = W.make_problem(nx, ny, nz, (10e-9, 12e-9, 9e-9), mask, alpha=0.05, Ku=2e3, ku_axis=ku,
                       B0=(0.01, 0.02, 0.18), Nd=(0.2, 0.3, 0.5),
                       omega=TP * np.array([5.0e9, 5.3e9]), kappa=TP * np.array([3e6, 8e6]),
                       g_re=TP * np.array([60e6, 40e6]), g_im=TP * np.array([10e6, -15e6]),
                       u=u, a0=np.array([0.01 + 0.004j, -0.003j]))
    m = W.random_state(1, nx, ny, nz, seed, spread=0.4) * mask
    return p.replace(m0=m)


def afm_case(seed=2):
    """Two-sublattice magnet with demag, inter-sublattice exchange and one profiled mode."""
    nx, ny, nz = 5, 4, 3
    mask = W.random_mask(nx, ny, nz, 0.85, seed)
    u = W.fourier_profiles(1, nx, ny, nz, seed + 3).astype(np.float64)
    p = W.make_problem(nx, ny, nz, 8e-9, mask, nsub=2, alpha=0.02, Ku=1e3, B0=(0.0, 0.05, 0.3),
                       Nd=(0.1, 0.1, 0.8), BE=1.5, omega=TP * np.array([20e9]),
                       kappa=TP * np.array([5e6]), g_re=TP * np.array([80e6]),
                       g_im=TP * np.array([5e6]), u=u, a0=np.array([0.02 - 0.01j]))
    m = W.random_state(2, nx, ny, nz, seed, spread=0.3, afm=True) * mask
    return p.replace(m0=m)


CASES = {"ferro": ferro_case, "afm": afm_case}


def flat_m(p):
    return np.asarray(p.m0, np.float64).reshape(-1).copy()


def masked_random(p, rng, scale=1.0):
    v = rng.normal(size=(p.nsub, 3, p.nz, p.ny, p.nx)) * p.mask.astype(float)
    return scale * v.reshape(-1)


def perturbed(p, name, idx, delta):
    """Copy of p with one parameter moved by delta (u: idx = (mode, flat cell))."""
    if name == "alpha":
        return p.replace(alpha=p.alpha + delta)
    if name == "u":
        u = np.array(p.u, np.float64).reshape(p.nmodes, -1).copy()
        u[idx] += delta
        return p.replace(u=u.reshape(p.u.shape))
    arr = np.array(getattr(p, name), np.float64).copy()
    arr[idx] += delta
    return p.replace(**{name: arr})


def param_value(p, name, idx):
    if name == "alpha":
        return p.alpha
    if name == "u":
        return float(np.asarray(p.u).reshape(p.nmodes, -1)[idx])
    return float(np.asarray(getattr(p, name))[idx])


def grad_entry(g, name, idx):
    if name == "alpha":
        return g["alpha"]
    if name == "u":
        return g["u"][idx]
    return g[name][idx]


def param_list(p, rng):
    cells = np.flatnonzero(p.mask.reshape(-1))
    out = []
    for n in range(p.nmodes):
        for name in ("g_re", "g_im", "kappa", "omega"):
            out.append((name, n))
        for c in rng.choice(cells, 2, replace=False):
            out.append(("u", (n, int(c))))
    out.append(("alpha", None))
    return out


def rel_step(name, value):
    if name == "u":
        return 1e-4
    return 1e-4 * max(abs(value), 1e6 if name != "alpha" else 1e-3)


def traj_step(name, value):
    """Central-difference steps for whole trajectories: large enough that the rounding noise of
    two replays (about 1e-16 of the loss terms) stays far below the truncation error, small
    enough (omega sets phases) that the truncation error stays below 1e-6 relative."""
    if name == "u":
        return 1e-2
    if name in ("omega", "alpha"):
        return 1e-4 * max(abs(value), 1e-3)
    return 1e-2 * max(abs(value), 1e6)


# ----------------------------------------------------------------------------------------------
# right-hand side: <w, J v> by central differences against <J^T w, v>
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", list(CASES))
def test_rhs_vjp_state_directional(case):
    p = CASES[case]()
    op = O.OracleProblem(p)
    rng = np.random.default_rng(11)
    m = flat_m(p)
    a = O.pack_a(p.a0)
    wm = masked_random(p, rng)
    wa = rng.normal(size=2 * p.nmodes) * 1e9
    vm = masked_random(p, rng)
    va = rng.normal(size=2 * p.nmodes) * 1e-2
    g = O.rhs_vjp(op, m, a, wm, wa)
    an = g["m"] @ vm + g["a"] @ va

    def dphi(vm_, va_, e):
        dmp, dap, _ = O.rhs(op, m + e * vm_, a + e * va_)
        dmn, dan, _ = O.rhs(op, m - e * vm_, a - e * va_)
        return (wm @ (dmp - dmn) + wa @ (dap - dan)) / (2 * e)

    eps = 1e-5
    fd = dphi(vm, va, eps)
    assert abs(fd - an) <= 1e-7 * abs(an), (fd, an)
    # each block alone, so no two mistakes can cancel
    for vm_, va_ in ((vm, 0 * va), (0 * vm, va)):
        an1 = g["m"] @ vm_ + g["a"] @ va_
        fd1 = dphi(vm_, va_, eps)
        assert abs(fd1 - an1) <= 1e-7 * abs(an1), (fd1, an1)


@pytest.mark.parametrize("case", list(CASES))
def test_rhs_vjp_parameters(case):
    p = CASES[case]()
    rng = np.random.default_rng(5)
    m = flat_m(p)
    a = O.pack_a(p.a0)
    wm = masked_random(p, rng)
    wa = rng.normal(size=2 * p.nmodes) * 1e9
    g = O.rhs_vjp(O.OracleProblem(p), m, a, wm, wa)
    for name, idx in param_list(p, rng):
        h = rel_step(name, param_value(p, name, idx))

        # difference the slopes elementwise before weighting (the weighted sums are large)
        dmp, dap, _ = O.rhs(O.OracleProblem(perturbed(p, name, idx, h)), m, a)
        dmn, dan, _ = O.rhs(O.OracleProblem(perturbed(p, name, idx, -h)), m, a)
        fd = (wm @ (dmp - dmn) + wa @ (dap - dan)) / (2 * h)
        an = grad_entry(g, name, idx)
        assert abs(fd - an) <= 1e-6 * max(abs(an), abs(fd)) + 1e-12, (name, idx, fd, an)


# ----------------------------------------------------------------------------------------------
# whole replayed step sequences
# ----------------------------------------------------------------------------------------------
def step_sizes(p, n):
    """The first n accepted step sizes of the oracle's own adaptive run."""
    it = O.Integrator(O.OracleProblem(p))
    rc, log = it.run(1.0, max_attempts=4 * n, log_cap=4 * n)
    v = log.view()
    dts = v["dt"][v["accepted"]][:n]
    assert len(dts) == n
    return dts


def loss_weights(p, n, rng):
    """A loss touching every state: L = sum_i <c_i, a_i> + |a_n,0|^2 + <wm, m_n>."""
    c = rng.normal(size=(n + 1, 2 * p.nmodes))
    wm = masked_random(p, rng)
    return c, wm


def loss_parts(p, dts, m0=None, a0=None):
    """Cavity states a_0..a_n (packed) and m_n of a replay."""
    op = O.OracleProblem(p)
    a0 = O.pack_a(p.a0) if a0 is None else a0
    it = O.Integrator(op, m=flat_m(p) if m0 is None else m0, a=a0)
    rc, log = it.replay(dts)
    assert rc == 0
    traj = np.concatenate([a0[None], np.stack([O.pack_a(x) for x in log.view()["a"]])])
    return traj, it.state()["m"]


def loss_difference(p_plus, p_minus, dts, c, wm, plus=(None, None), minus=(None, None)):
    """L(+) - L(-), differenced term by term before weighting (the sums are large)."""
    tp, mp = loss_parts(p_plus, dts, *plus)
    tn, mn = loss_parts(p_minus, dts, *minus)
    quad = (tp[-1, 0] - tn[-1, 0]) * (tp[-1, 0] + tn[-1, 0]) + \
        (tp[-1, 1] - tn[-1, 1]) * (tp[-1, 1] + tn[-1, 1])
    return float(np.sum(c * (tp - tn)) + quad + wm @ (mp - mn))


def loss_grads(p, dts, c, wm):
    op = O.OracleProblem(p)
    it = O.Integrator(op)
    rc, _ = it.replay(dts)
    aT = O.pack_a(it.state()["a"])
    dL_da = c.copy()
    dL_da[-1, 0] += 2 * aT[0]
    dL_da[-1, 1] += 2 * aT[1]
    return O.adjoint(op, flat_m(p), O.pack_a(p.a0), dts, dL_da, wm)


@pytest.mark.parametrize("case,nsteps", [("ferro", 25), ("afm", 15)])
def test_adjoint_parameters_match_central_differences(case, nsteps):
    p = CASES[case]()
    rng = np.random.default_rng(9)
    dts = step_sizes(p, nsteps)
    c, wm = loss_weights(p, nsteps, rng)
    g = loss_grads(p, dts, c, wm)
    for name, idx in param_list(p, rng):
        h = traj_step(name, param_value(p, name, idx))
        fd = loss_difference(perturbed(p, name, idx, h), perturbed(p, name, idx, -h), dts, c,
                             wm) / (2 * h)
        an = grad_entry(g, name, idx)
        assert abs(fd - an) <= 2e-6 * max(abs(an), abs(fd)) + 1e-14, (name, idx, fd, an)


@pytest.mark.parametrize("case,nsteps", [("ferro", 25), ("afm", 15)])
def test_adjoint_initial_state_matches_central_differences(case, nsteps):
    p = CASES[case]()
    rng = np.random.default_rng(4)
    dts = step_sizes(p, nsteps)
    c, wm = loss_weights(p, nsteps, rng)
    g = loss_grads(p, dts, c, wm)
    m0, a0 = flat_m(p), O.pack_a(p.a0)
    cells = np.flatnonzero(np.abs(m0) > 0)
    for i in list(rng.choice(cells, 4, replace=False)):
        e = np.zeros_like(m0)
        e[i] = 1e-6
        fd = loss_difference(p, p, dts, c, wm, (m0 + e, None), (m0 - e, None)) / 2e-6
        assert abs(fd - g["m0"][i]) <= 2e-6 * abs(fd) + 1e-10, (i, fd, g["m0"][i])
    for q in range(2 * p.nmodes):
        e = np.zeros_like(a0)
        e[q] = 1e-6
        fd = loss_difference(p, p, dts, c, wm, (None, a0 + e), (None, a0 - e)) / 2e-6
        assert abs(fd - g["a0"][q]) <= 2e-6 * abs(fd) + 1e-10, (q, fd, g["a0"][q])


def test_free_cavity_decay_closed_form():
    """g = 0: |a(T)|^2 = |a0|^2 exp(-2 kappa T), so dL/dkappa = -2 T L and dL/domega = 0."""
    nx = ny = nz = 3
    p = W.make_problem(nx, ny, nz, 10e-9, W.full_mask(nx, ny, nz), B0=(0, 0, 0.2),
                       omega=[TP * 5e9], kappa=[TP * 20e6], g_re=[0.0], g_im=[0.0],
                       a0=np.array([0.01 + 0.002j]), rtol=1e-9)
    op = O.OracleProblem(p)
    T = 5e-9
    it = O.Integrator(op)
    rc, log = it.run(T, log_cap=200000)
    v = log.view()
    dts = v["dt"][v["accepted"]]
    aT = O.pack_a(it.state()["a"])
    L = aT @ aT
    dL_da = np.zeros((len(dts) + 1, 2))
    dL_da[-1] = 2 * aT
    g = O.adjoint(op, flat_m(p), O.pack_a(p.a0), dts, dL_da, None)
    assert abs(L - abs(p.a0[0]) ** 2 * math.exp(-2 * p.kappa[0] * T)) <= 1e-7 * L
    assert abs(g["kappa"][0] - (-2 * T * L)) <= 1e-6 * abs(2 * T * L)
    assert abs(g["omega"][0]) <= 1e-6 * abs(2 * T * L)
    # the initial amplitude: L = |a0|^2 exp(-2 kappa T)  ->  dL/da0 = 2 a0 exp(-2 kappa T)
    want = 2 * O.pack_a(p.a0) * math.exp(-2 * p.kappa[0] * T)
    assert np.allclose(g["a0"], want, rtol=1e-7, atol=0)
