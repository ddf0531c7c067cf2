"""Pins of the oracle's cavity-model extensions (CPU only): nonreciprocal coupling (a backward
coefficient gb~ for the feedback field, Sec. II: h0 = 2 g_b / gamma) and a self-Kerr term
-i K |a|^2 a in the cavity equation.

* Linearised about the ground state, a macrospin coupled nonreciprocally has exactly the
  eigenvalues of the hand-derived Kittel + cavity matrix with g_f in the cavity row and g_b in
  the magnet row; their product replaces g^2 in the branches of Eq. (6).
* A free Kerr cavity keeps |a| = |a0| e^{-kappa t} and turns its phase at w + K |a|^2:
  theta(t) = theta0 - w t - K |a0|^2 (1 - e^{-2 kappa t}) / (2 kappa).
* The adjoint's gradients with respect to gb~ and K match central differences.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import workloads as W

from test_oracle_pins import G, nearest, spectrum

TP = 2 * math.pi


def nonreciprocal_matrix(wm, alpha, w, k, gf, gb):
    """Hand-linearised Kittel mode + one cavity (variables m-, conj m-, a, conj a): the feedback
    field B_x = (1/gamma)(gb~ a + conj(gb~ a)) drives the magnet, i gf~ m- drives the cavity."""
    M = np.zeros((4, 4), complex)
    cm = -(alpha + 1j) * wm
    M[0, 0], M[1, 1] = cm, np.conj(cm)
    fac = (alpha + 1j) / (1 + alpha ** 2)
    M[0, 2], M[0, 3] = fac * gb, fac * np.conj(gb)
    M[1, 2], M[1, 3] = np.conj(fac) * gb, np.conj(fac) * np.conj(gb)
    M[2, 2], M[3, 3] = -1j * w - k, 1j * w - k
    M[2, 0], M[3, 1] = 1j * gf, np.conj(1j * gf)
    return M


@pytest.mark.parametrize("gf_MHz,gb_MHz", [(50.0, 20.0), (30.0, 80.0 + 10.0j), (50.0, -40.0)])
def test_nonreciprocal_linearisation(gf_MHz, gb_MHz):
    p = W.single_sphere()
    gf, gb = TP * 1e6 * complex(gf_MHz), TP * 1e6 * complex(gb_MHz)
    p = p.replace(g_re=np.array([gf.real]), g_im=np.array([gf.imag]), g_back=np.array([gb]))
    ev = spectrum(p)
    wm = G * p.B0[2] / (1 + p.alpha ** 2)
    M = nonreciprocal_matrix(wm, p.alpha, p.omega[0], p.kappa[0], gf, gb)
    for lam in np.linalg.eigvals(M):
        assert abs(nearest(ev, lam) - lam) < 1e-8 * abs(lam)


def test_nonreciprocal_branches_use_the_product_of_couplings():
    """At resonance the splitting is 2 sqrt(g_f g_b) (Eq. (6) with g^2 -> g_f g_b)."""
    p = W.single_sphere()
    gf, gb = TP * 80e6, TP * 20e6
    p = p.replace(g_re=np.array([gf]), g_im=np.array([0.0]), g_back=np.array([gb + 0j]))
    ev = spectrum(p)
    wc = p.omega[0]
    for sgn in (+1, -1):
        w = wc + sgn * math.sqrt(gf * gb)
        lam = nearest(ev, -1j * w)
        assert abs(-lam.imag - w) < TP * 0.2e6


@pytest.mark.parametrize("K", [TP * 5e9, -TP * 2e9])
def test_kerr_free_cavity_closed_form(K):
    n = 2
    a0 = 0.03 + 0.01j
    p = W.make_problem(n, n, n, 10e-9, W.full_mask(n, n, n), B0=(0, 0, 0.2),
                       omega=[TP * 5.0e9], kappa=[TP * 30e6], g_re=[0.0], g_im=[0.0],
                       a0=np.array([a0]), rtol=1e-11, dt_max=2e-12).replace(
                           kerr=np.array([K]))
    T = 1.5e-9
    it = O.Integrator(O.OracleProblem(p))
    rc, _ = it.run(T)
    assert rc == 0
    a = it.state()["a"][0]
    k, w = p.kappa[0], p.omega[0]
    r0, th0 = abs(a0), np.angle(a0)
    th = th0 - w * T - K * r0 ** 2 * (1 - math.exp(-2 * k * T)) / (2 * k)
    want = r0 * math.exp(-k * T) * np.exp(1j * th)
    assert abs(a - want) <= 1e-8 * abs(want), (a, want)


def test_adjoint_backward_coupling_and_kerr_gradients():
    nx, ny, nz = 5, 4, 3
    mask = W.random_mask(nx, ny, nz, 0.85, 6)
    p = W.make_problem(nx, ny, nz, 10e-9, mask, alpha=0.02, B0=(0, 0, TP * 5e9 / W.GAMMA),
                       Nd=(0.2, 0.3, 0.5), omega=TP * np.array([5.0e9, 5.2e9]),
                       kappa=TP * np.array([5e6, 3e6]), g_re=TP * np.array([80e6, 40e6]),
                       g_im=TP * np.array([10e6, 0.0]), u=W.fourier_profiles(2, nx, ny, nz, 1),
                       m0=W.random_state(1, nx, ny, nz, 7, spread=0.3) * mask,
                       a0=np.array([0.02 + 0.01j, -0.015j]))
    p = p.replace(g_back=TP * np.array([30e6 + 5e6j, 60e6 - 10e6j]),
                  kerr=TP * np.array([3e9, -1e9]))
    op = O.OracleProblem(p)
    dts = np.full(25, 2e-12)
    rng = np.random.default_rng(2)
    c = rng.normal(size=(26, 4))

    def traj(q):
        it = O.Integrator(O.OracleProblem(q))
        rc, log = it.replay(dts)
        return np.concatenate([O.pack_a(q.a0)[None],
                               np.stack([O.pack_a(x) for x in log.view()["a"]])])

    g = O.adjoint(op, op.m0(), O.pack_a(p.a0), dts, c, None)
    cases = [("gb", 0, 1.0), ("gb", 1, 1j), ("kerr", 0, None), ("kerr", 1, None)]
    for name, n, direction in cases:
        if name == "gb":
            h = 1e-3 * abs(p.g_back[n])
            gp, gm = p.g_back.copy(), p.g_back.copy()
            gp[n] += h * direction
            gm[n] -= h * direction
            qp, qm = p.replace(g_back=gp), p.replace(g_back=gm)
            an = g["gb_re"][n] if direction == 1.0 else g["gb_im"][n]
        else:
            h = 1e-3 * abs(p.kerr[n])
            kp, km = p.kerr.copy(), p.kerr.copy()
            kp[n] += h
            km[n] -= h
            qp, qm = p.replace(kerr=kp), p.replace(kerr=km)
            an = g["kerr"][n]
        fd = float(np.sum(c * (traj(qp) - traj(qm)))) / (2 * h)
        assert abs(fd - an) <= 1e-5 * abs(fd), (name, n, fd, an)
    # the Kerr Jacobian's transpose, through the initial amplitudes
    a0 = O.pack_a(p.a0)
    for q in range(4):
        e = np.zeros(4)
        e[q] = 1e-6

        def tr_a0(av):
            it = O.Integrator(op, a=av)
            rc, log = it.replay(dts)
            return np.concatenate([av[None], np.stack([O.pack_a(x) for x in log.view()["a"]])])

        fd = float(np.sum(c * (tr_a0(a0 + e) - tr_a0(a0 - e)))) / 2e-6
        assert abs(fd - g["a0"][q]) <= 1e-6 * abs(fd), (q, fd, g["a0"][q])
