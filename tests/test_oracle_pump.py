"""Pins of the oracle's parametric pump (CPU only).  The paper names parametric drives as a
cavity-model swap (Sec. V) without a formula; the oracle's reading is the classical equation of
a degenerate two-photon pump, da_n/dt += -i P_n e^{-i wp_n t} conj(a_n).

* In the frame b = a e^{i wp t / 2} a free pumped cavity obeys the autonomous linear system
  db/dt = (i D - kappa) b - i P conj(b), D = wp/2 - w.  Its 2 x 2 real matrix M satisfies
  (M + kappa)^2 = (|P|^2 - D^2) I, so exp(M tau) = e^{-kappa tau} [cosh(l tau) I +
  sinh(l tau)/l (M + kappa)], l = sqrt(|P|^2 - D^2): the textbook threshold |P|^2 = kappa^2 +
  D^2 of parametric oscillation.  Checked on resonance (D = 0, below and above threshold), off
  resonance (oscillating), with a complex P and a start time t0 != 0 (the pump phase is
  referenced to t = 0).
* The operator-split run (classical RK4 for the cavity) converges to the same closed form at
  fourth order when the magnet is decoupled.
* The adjoint's gradients with respect to Re P and Im P match central differences of the
  replayed trajectory, and its gradient with respect to the initial amplitudes (through the
  pump's Jacobian transpose) matches central differences too.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import workloads as W

TP = 2 * math.pi


def pumped_cavity(a0, w, k, P, wp, t0, t):
    """Closed form of the free pumped cavity from a(t0) = a0 (see the module docstring)."""
    D = 0.5 * wp - w
    b0 = a0 * np.exp(0.5j * wp * t0)
    x = np.array([b0.real, b0.imag])
    Pr, Pi = P.real, P.imag
    # -i P conj(b) = (Pi br - Pr bi) - i (Pr br + Pi bi)
    Mk = np.array([[Pi, -D - Pr], [D - Pr, -Pi]])     # M + kappa I
    lam = np.sqrt(complex(abs(P) ** 2 - D * D))
    tau = t - t0
    ch = np.cosh(lam * tau).real
    sh = (np.sinh(lam * tau) / lam).real if abs(lam) > 0 else tau
    y = math.exp(-k * tau) * (ch * x + sh * (Mk @ x))
    return complex(y[0], y[1]) * np.exp(-0.5j * wp * t)


def free_cavity_problem(w, k, P, wp, a0, **kw):
    n = 2
    p = W.make_problem(n, n, n, 10e-9, W.full_mask(n, n, n), B0=(0, 0, 0.2), omega=[w],
                       kappa=[k], g_re=[0.0], g_im=[0.0], a0=np.array([a0]), **kw)
    return p.replace(pump=np.array([P]), pump_omega=np.array([wp]))


def test_closed_form_matrix_identity():
    """(M + kappa)^2 = (|P|^2 - D^2) I for the matrix used by the closed form."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        D, Pr, Pi = rng.normal(size=3)
        Mk = np.array([[Pi, -D - Pr], [D - Pr, -Pi]])
        assert np.allclose(Mk @ Mk, (Pr * Pr + Pi * Pi - D * D) * np.eye(2), atol=1e-12)


@pytest.mark.parametrize("eps_over_kappa,phase,detune_MHz,t0", [
    (0.5, 0.0, 0.0, 0.0),          # below threshold: both quadratures decay
    (3.0, 0.0, 0.0, 0.0),          # above threshold: one quadrature grows at eps - kappa
    (2.0, 0.7, 0.0, 0.31e-9),      # complex pump, start time != 0
    (1.5, -1.1, 90.0, 0.17e-9),    # detuned beyond threshold: oscillating
    (4.0, 0.3, 40.0, 0.0),         # detuned, still amplifying
])
def test_free_pumped_cavity_closed_form(eps_over_kappa, phase, detune_MHz, t0):
    w, k = TP * 5.0e9, TP * 30e6
    P = eps_over_kappa * k * np.exp(1j * phase)
    wp = 2 * (w + TP * detune_MHz * 1e6)
    a0 = 0.03 + 0.01j
    p = free_cavity_problem(w, k, P, wp, a0, rtol=1e-11, dt_max=2e-12)
    T = t0 + 1.5e-9
    it = O.Integrator(O.OracleProblem(p), t0=t0)
    rc, _ = it.run(T)
    assert rc == 0
    a = it.state()["a"][0]
    want = pumped_cavity(a0, w, k, P, wp, t0, T)
    assert abs(a - want) <= 1e-8 * abs(want), (a, want)


def test_threshold_growth_rate():
    """Above threshold on resonance the amplitude grows at eps - kappa: |a(T2)| / |a(T1)| for
    late times approaches e^{(eps - kappa)(T2 - T1)}."""
    w, k = TP * 5.0e9, TP * 30e6
    eps = 2.5 * k
    p = free_cavity_problem(w, k, eps, 2 * w, 0.01 + 0.0j, rtol=1e-10, dt_max=2e-12)
    it = O.Integrator(O.OracleProblem(p))
    rc, _ = it.run(20e-9)
    assert rc == 0
    a1 = it.state()["a"][0]
    rc, _ = it.run(25e-9)
    assert rc == 0
    a2 = it.state()["a"][0]
    rate = math.log(abs(a2) / abs(a1)) / 5e-9
    assert abs(rate - (eps - k)) <= 1e-6 * (eps - k)


def test_split_rk4_converges_to_closed_form():
    w, k = TP * 5.0e9, TP * 30e6
    P = 2.0 * k * np.exp(0.4j)
    wp = 2 * (w + TP * 20e6)
    a0 = 0.02 - 0.01j
    p = free_cavity_problem(w, k, P, wp, a0, rtol=1e-9, dt_max=2e-12)
    T = 0.4e-9
    want = pumped_cavity(a0, w, k, P, wp, 0.0, T)
    errs = []
    for ds in (8e-12, 4e-12, 2e-12):
        it = O.Integrator(O.OracleProblem(p))
        rc, _ = it.run_split(T, ds)
        assert rc == 0
        errs.append(abs(it.state()["a"][0] - want))
    order = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.7 < o < 4.3 for o in order), (errs, order)


def test_adjoint_pump_gradients():
    nx, ny, nz = 5, 4, 3
    mask = W.random_mask(nx, ny, nz, 0.85, 6)
    p = W.make_problem(nx, ny, nz, 10e-9, mask, alpha=0.02, B0=(0, 0, TP * 5e9 / W.GAMMA),
                       Nd=(0.2, 0.3, 0.5), omega=TP * np.array([5.0e9, 5.2e9]),
                       kappa=TP * np.array([5e6, 3e6]), g_re=TP * np.array([80e6, 40e6]),
                       g_im=TP * np.array([10e6, 0.0]), u=W.fourier_profiles(2, nx, ny, nz, 1),
                       m0=W.random_state(1, nx, ny, nz, 7, spread=0.3) * mask,
                       a0=np.array([0.02 + 0.01j, -0.015j]))
    p = p.replace(pump=TP * np.array([20e6 + 5e6j, -8e6 + 12e6j]),
                  pump_omega=TP * np.array([10.02e9, 10.4e9]))
    t0 = 0.37e-9
    op = O.OracleProblem(p)
    dts = np.full(25, 2e-12)
    rng = np.random.default_rng(2)
    c = rng.normal(size=(26, 4))

    def traj(q, av=None):
        it = O.Integrator(O.OracleProblem(q), a=av, t0=t0)
        rc, log = it.replay(dts)
        assert rc == 0
        first = O.pack_a(q.a0) if av is None else av
        return np.concatenate([first[None], np.stack([O.pack_a(x) for x in log.view()["a"]])])

    g = O.adjoint(op, op.m0(), O.pack_a(p.a0), dts, c, None, t0=t0)
    assert np.abs(g["pump_re"]).max() > 0 and np.abs(g["pump_im"]).max() > 0
    for n in range(2):
        for direction, key in ((1.0, "pump_re"), (1j, "pump_im")):
            h = 1e-3 * abs(p.pump[n])
            pp, pm = p.pump.copy(), p.pump.copy()
            pp[n] += h * direction
            pm[n] -= h * direction
            fd = float(np.sum(c * (traj(p.replace(pump=pp)) - traj(p.replace(pump=pm))))) / (2 * h)
            assert abs(fd - g[key][n]) <= 1e-5 * abs(fd), (key, n, fd, g[key][n])
    a0 = O.pack_a(p.a0)
    for q in range(4):
        e = np.zeros(4)
        e[q] = 1e-6
        fd = float(np.sum(c * (traj(p, a0 + e) - traj(p, a0 - e)))) / 2e-6
        assert abs(fd - g["a0"][q]) <= 1e-6 * abs(fd), (q, fd, g["a0"][q])
