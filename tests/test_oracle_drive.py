"""Pins of the oracle's external drive eta_n(t) (Eq. (1), (12); Gaussian pulse of Sec. IV A),
CPU only.

* A cavity without magnet coupling is a damped oscillator driven by a Gaussian: its amplitude has
  a closed form in the complex error function,
      a(t) = e^{lam t} [ a0 + eta0 sigma sqrt(pi/2) e^{lam^2 sigma^2 / 2 - lam t0}
                         (erf((t - mu) / (sqrt2 sigma)) + erf(mu / (sqrt2 sigma))) ],
  lam = -i w - kappa, mu = t0 - lam sigma^2 (completing the square in the Duhamel integral).
* Replays with steps h and h/2 converge at fifth order, which only holds if every stage sees the
  drive at its own time t + c_s h.
* The discrete adjoint of a driven run still matches central differences.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

from oracle import oracle as O
from paper_2603_03706_b300 import workloads as W

TP = 2 * math.pi


def free_cavity(drive, t0=0.1e-9, sigma=20e-12, a0=(0.0, 0.0), rtol=1e-11):
    n = 3
    return W.make_problem(n, n, n, 10e-9, W.full_mask(n, n, n), B0=(0, 0, 0.2),
                          omega=TP * np.array([5.0e9, 5.3e9]), kappa=TP * np.array([3e6, 40e6]),
                          g_re=[0.0, 0.0], g_im=[0.0, 0.0], a0=np.array(a0, complex),
                          rtol=rtol, dt_max=2e-12).replace(drive=np.asarray(drive, complex),
                                                           drive_t0=t0, drive_sigma=sigma)


def closed_form(p, t):
    lam = -1j * p.omega - p.kappa
    s, t0 = p.drive_sigma, p.drive_t0
    mu = t0 - lam * s * s
    r2 = math.sqrt(2.0) * s
    integral = s * math.sqrt(math.pi / 2) * np.exp(lam * lam * s * s / 2 - lam * t0) * (
        erf((t - mu) / r2) + erf(mu / r2))
    return np.exp(lam * t) * (np.asarray(p.a0, complex) + np.asarray(p.drive) * integral)


@pytest.mark.parametrize("T", [0.05e-9, 0.1e-9, 0.3e-9, 2e-9])
def test_driven_free_cavity_closed_form(T):
    p = free_cavity(drive=[3e7 + 1e7j, -2e7j], a0=(1e-3 + 2e-4j, 0))
    it = O.Integrator(O.OracleProblem(p))
    rc, _ = it.run(T)
    assert rc == 0
    a = it.state()["a"]
    want = closed_form(p, T)
    assert np.abs(a - want).max() <= 1e-8 * np.abs(want).max(), (a, want)


def test_drive_stage_times_give_fifth_order():
    p = free_cavity(drive=[3e7, 1e7j])
    T = 0.2e-9
    errs = []
    for n in (40, 80):
        it = O.Integrator(O.OracleProblem(p))
        rc, _ = it.replay(np.full(n, T / n), log=False)
        assert rc == 0
        errs.append(np.abs(it.state()["a"] - closed_form(p, T)).max())
    ratio = errs[0] / errs[1]
    assert 20.0 < ratio < 45.0, (errs, ratio)   # 2^5 = 32


def test_drive_starts_where_the_run_starts():
    """Shifting the start time and the pulse centre together changes nothing."""
    dts = np.full(60, 4e-12)
    res = []
    for shift in (0.0, 0.37e-9):
        p = free_cavity(drive=[2e7 - 1e7j, 3e7], t0=0.1e-9 + shift)
        it = O.Integrator(O.OracleProblem(p), t0=shift)
        rc, _ = it.replay(dts, log=False)
        assert rc == 0
        res.append(it.state()["a"])
    assert np.abs(res[0] - res[1]).max() <= 1e-12 * np.abs(res[0]).max()


def test_adjoint_of_a_driven_coupled_run():
    nx, ny, nz = 5, 4, 3
    mask = W.random_mask(nx, ny, nz, 0.85, 5)
    p = W.make_problem(nx, ny, nz, 10e-9, mask, alpha=0.02, B0=(0, 0, TP * 5e9 / W.GAMMA),
                       Nd=(0.2, 0.3, 0.5), omega=[TP * 5.0e9], kappa=[TP * 5e6],
                       g_re=[TP * 80e6], g_im=[TP * 10e6], u=W.fourier_profiles(1, nx, ny, nz, 2),
                       m0=W.random_state(1, nx, ny, nz, 3, spread=0.2) * mask)
    p = p.replace(drive=np.array([5e7 + 2e7j]), drive_t0=30e-12, drive_sigma=10e-12)
    op = O.OracleProblem(p)
    dts = np.full(30, 2e-12)
    t_start = 5e-12
    it = O.Integrator(op, t0=t_start)
    rc, log = it.replay(dts)
    aT = O.pack_a(it.state()["a"])
    la = np.zeros((31, 2))
    la[-1] = 2 * aT
    g = O.adjoint(op, op.m0(), O.pack_a(p.a0), dts, la, None, t0=t_start)

    def L(q):
        it = O.Integrator(O.OracleProblem(q), t0=t_start)
        it.replay(dts, log=False)
        a = it.state()["a"]
        return float(np.abs(a[0]) ** 2)

    for name in ("g_re", "kappa", "omega"):
        v = np.array(getattr(p, name), float)
        h = (1e-2 if name != "omega" else 1e-5) * abs(v[0])
        vp, vm = v.copy(), v.copy()
        vp[0] += h
        vm[0] -= h
        fd = (L(p.replace(**{name: vp})) - L(p.replace(**{name: vm}))) / (2 * h)
        assert abs(fd - g[name][0]) <= 1e-5 * abs(fd), (name, fd, g[name][0])
