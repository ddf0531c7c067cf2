"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one part of the oracle to something other than the oracle itself: a closed form
from the paper (Kittel, polariton branches, AFMR, Rabi period, dark mode, level attraction), a
textbook result (Neumann Laplacian spectrum, macrospin damping, Butcher order conditions), a
library computation (graph Laplacian, scipy's DOP853), or a value printed in the paper
(tests/golden/).  A dropped term, a wrong sign or a transposed index in the oracle breaks at
least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
G = W.GAMMA
TP = 2 * math.pi


def read_golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


def uniform_z(p, afm=False):
    mask = p.mask.astype(float)
    m = np.zeros((p.nsub, 3, p.nz, p.ny, p.nx))
    m[0, 2] = mask
    if p.nsub == 2:
        m[1, 2] = -mask if afm else mask
    return m.reshape(-1)


def spectrum(p, m=None, a=None):
    op = O.OracleProblem(p)
    if m is None:
        m = uniform_z(p, afm=p.nsub == 2)
    if a is None:
        a = np.zeros(2 * p.nmodes)
    J, _ = O.jacobian(op, m, a)
    return np.linalg.eigvals(J)


def nearest(ev, target):
    return ev[np.argmin(np.abs(ev - target))]


# ------------------------------------------------------------------------------------------
# Dormand-Prince tableau: Butcher order conditions (order 5 for b5, order 4 for b4)
# ------------------------------------------------------------------------------------------

def _trees(n, memo={}):
    """All rooted trees with n vertices as sorted tuples of child subtrees."""
    if n in memo:
        return memo[n]
    if n == 1:
        memo[1] = [()]
        return memo[1]
    out = set()

    def parts(rem, maxsize, acc):
        if rem == 0:
            yield tuple(sorted(acc))
            return
        for s in range(min(rem, maxsize), 0, -1):
            for t in _trees(s):
                yield from parts(rem - s, s, acc + [t])
    for forest in parts(n - 1, n - 1, []):
        out.add(forest)
    memo[n] = sorted(out)
    return memo[n]


def _order(t):
    return 1 + sum(_order(c) for c in t)


def _density(t):
    return _order(t) * math.prod(_density(c) for c in t)


def _weights(t, A):
    v = np.ones(A.shape[0])
    for c in t:
        v = v * (A @ _weights(c, A))
    return v


def test_tableau_order_conditions():
    a6, b5, b4 = O.tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a6
    c = A.sum(axis=1)
    assert np.allclose(c, [0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1, 1], atol=1e-15)
    assert np.allclose(A[6], b5, atol=1e-16)          # first-same-as-last
    nconds = 0
    for order in range(1, 6):
        for t in _trees(order):
            target = 1.0 / _density(t)
            assert abs(b5 @ _weights(t, A) - target) < 1e-14, (order, t)
            if order <= 4:
                assert abs(b4 @ _weights(t, A) - target) < 1e-14, (order, t)
            nconds += 1
    assert nconds == 17
    # the embedded pair differs at order 5 (otherwise the error estimate would vanish)
    t5 = _trees(5)
    assert max(abs(b4 @ _weights(t, A) - 1 / _density(t)) for t in t5) > 1e-4


# ------------------------------------------------------------------------------------------
# local field and torque: Kittel, Neumann Laplacian, demag, anisotropy, AFMR
# ------------------------------------------------------------------------------------------

def test_torque_is_perpendicular_to_m():
    """dm/dt from the LLG torque is orthogonal to m in every cell, so |m| = 1 is conserved."""
    p = W.make_problem(5, 4, 3, 5e-9, W.random_mask(5, 4, 3, 0.7, 1), Ku=300.0,
                       ku_axis=(0.6, 0, 0.8), B0=(0.01, -0.02, 0.2), Nd=(0.2, 0.3, 0.5),
                       omega=[TP * 5e9], kappa=[TP * 5e6], g_re=[TP * 50e6], g_im=[TP * 20e6],
                       u=np.random.default_rng(0).uniform(-1, 1, (1, 3, 4, 5)))
    op = O.OracleProblem(p)
    m = W.random_state(1, 5, 4, 3, seed=2).reshape(-1)
    dm, _, _ = O.rhs(op, m, O.pack_a([0.003 - 0.002j]))
    m3, d3 = m.reshape(3, -1), dm.reshape(3, -1)
    dot = np.abs((m3 * d3).sum(0))
    assert dot.max() <= 1e-12 * np.abs(d3).max()


@pytest.mark.parametrize("Ku", [0.0, -610.0])
def test_kittel_sphere(Ku):
    """Uniform mode of a sphere (isotropic demag) at omega = gamma (B0 + 2 K_u / M_s), Eq. (9);
    decay rate alpha omega (Sec. II C) in the Landau-Lifshitz form."""
    alpha, B0 = 1e-3, 0.18
    p = W.make_problem(6, 6, 6, 5e-9, W.sphere_mask(6, 6, 6), alpha=alpha, Ku=Ku, B0=(0, 0, B0),
                       Nd=(1 / 3, 1 / 3, 1 / 3))
    ev = spectrum(p)
    w = G * (B0 + 2 * Ku / p.Ms) / (1 + alpha ** 2)
    lam = nearest(ev, -alpha * w - 1j * w)
    assert abs(lam - (-alpha * w - 1j * w)) < 1e-7 * w


def test_neumann_laplacian_spectrum_full_box():
    """Full box, no demag: every spin wave sits at gamma (B0 + (2A/Ms) sum_d (2/c_d^2)
    (1 - cos(p_d pi / N_d))), the exact spectrum of the free-surface discrete Laplacian."""
    nx, ny, nz = 4, 3, 2
    c = (4e-9, 5e-9, 6e-9)
    p = W.make_problem(nx, ny, nz, c, W.full_mask(nx, ny, nz), alpha=0.0, B0=(0, 0, 0.2))
    ev = spectrum(p)
    lam_ex = 2 * p.Aex / p.Ms
    want = []
    for px in range(nx):
        for py in range(ny):
            for pz in range(nz):
                s = sum(2 / cd ** 2 * (1 - math.cos(pd * math.pi / nd))
                        for pd, nd, cd in ((px, nx, c[0]), (py, ny, c[1]), (pz, nz, c[2])))
                want.append(G * (0.2 + lam_ex * s))
    got = np.sort(np.abs(ev.imag[ev.imag > 1.0]))
    assert len(got) == len(want)
    assert np.allclose(got, np.sort(want), rtol=1e-8)


def test_masked_exchange_is_graph_laplacian():
    """Irregular mask with holes: the spin-wave spectrum equals gamma (B0 + (2A/Ms) mu) for the
    eigenvalues mu of the weighted graph Laplacian of the mask's face-adjacency graph (built
    with networkx), i.e. neighbours outside the mask contribute nothing."""
    import networkx as nx_
    nx, ny, nz = 4, 4, 3
    c = (5e-9, 4e-9, 6e-9)
    mask = W.random_mask(nx, ny, nz, 0.65, seed=7)
    p = W.make_problem(nx, ny, nz, c, mask, alpha=0.0, B0=(0, 0, 0.15))
    Gr = nx_.Graph()
    cells = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx) if mask[z, y, x]]
    Gr.add_nodes_from(cells)
    for (x, y, z) in cells:
        for d, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            q = (x + dx, y + dy, z + dz)
            if q in Gr:
                Gr.add_edge((x, y, z), q, weight=1.0 / c[d] ** 2)
    L = nx_.laplacian_matrix(Gr, weight="weight").toarray()
    mu = np.linalg.eigvalsh(L)
    want = np.sort(G * (0.15 + 2 * p.Aex / p.Ms * mu))
    ev = spectrum(p)
    got = np.sort(np.abs(ev.imag[ev.imag > 1.0]))
    assert np.allclose(got, want, rtol=1e-8)


def test_demag_film_kittel():
    """Thin film, N = (0, 0, 1): perpendicular field gives omega = gamma (B0 - mu0 Ms);
    in-plane field gives omega = gamma sqrt(B0 (B0 + mu0 Ms)) (Kittel 1948, cited in Sec. II D)."""
    mu0Ms = W.MU0 * 1.4e5
    p = W.make_problem(1, 1, 1, 5e-9, W.full_mask(1, 1, 1), alpha=0.0, B0=(0, 0, 0.3),
                       Nd=(0, 0, 1))
    ev = spectrum(p, m=np.array([0, 0, 1.0]))
    assert abs(ev.imag.max() - G * (0.3 - mu0Ms)) < 1e-8 * G * 0.3
    p = p.replace(B0=np.array([0.05, 0, 0]))
    ev = spectrum(p, m=np.array([1.0, 0, 0]))
    assert abs(ev.imag.max() - G * math.sqrt(0.05 * (0.05 + mu0Ms))) < 1e-8 * G * 0.05


def test_macrospin_precession_and_damping_closed_form():
    """Single spin in B0 z: phi(t) = phi0 + gamma' B0 t and tan(theta/2) = tan(theta0/2)
    exp(-alpha gamma' B0 t), gamma' = gamma/(1+alpha^2).  The integrator (Dormand-Prince with
    renormalisation) reproduces it to the tolerance of its error control."""
    alpha, B0, th0 = 0.05, 0.2, math.radians(30)
    p = W.make_problem(1, 1, 1, 5e-9, W.full_mask(1, 1, 1), alpha=alpha, B0=(0, 0, B0),
                       rtol=1e-9, m0=np.array([math.sin(th0), 0, math.cos(th0)]).reshape(1, 3, 1, 1, 1))
    it = O.Integrator(O.OracleProblem(p))
    T = 0.4e-9
    rc, _ = it.run(T)
    assert rc == 0
    m = it.state()["m"]
    gp = G / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * gp * B0 * T))
    ph = gp * B0 * T
    want = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    assert np.abs(m - want).max() < 2e-7


def test_afmr_branches_with_exchange_spin_waves():
    """Two sublattices on a small film, field B along the easy axis: every spin wave sits at
    gamma (B +- sqrt((B_A + l_p)(2 B_E + B_A + l_p))) with l_p the exchange eigenvalue of the
    Neumann Laplacian; l_0 = 0 gives omega_AFMR +- gamma B, Eqs. (15)-(16).  Film demag
    (0, 0, 1) on the total moment drops out at linear order."""
    nx, ny, nz = 3, 2, 1
    c = 2e-9
    Ms, K, BE, B = 4e5, 5e4, 50.0, 1.0
    BA = 2 * K / Ms
    p = W.make_problem(nx, ny, nz, c, W.full_mask(nx, ny, nz), nsub=2, Ms=Ms, Aex=5e-12,
                       alpha=0.0, Ku=K, B0=(0, 0, B), Nd=(0, 0, 1), BE=BE)
    ev = spectrum(p)
    lam_ex = 2 * p.Aex / Ms
    want = []
    for px in range(nx):
        for py in range(ny):
            lp = lam_ex * (2 / c ** 2 * (1 - math.cos(px * math.pi / nx))
                           + 2 / c ** 2 * (1 - math.cos(py * math.pi / ny)))
            r = math.sqrt((BA + lp) * (2 * BE + BA + lp))
            want += [G * (r + B), G * (r - B)]
    got = np.sort(np.abs(ev.imag[ev.imag > 1.0]))
    assert np.allclose(got, np.sort(want), rtol=1e-7)
    # uniform branches equal Eq. (16)
    w_afmr = G * math.sqrt(2 * BE * BA + BA ** 2)
    assert abs(nearest(got, w_afmr - G * B) - (w_afmr - G * B)) < 1e-7 * w_afmr


def test_afmr_paper_parameters_golden():
    """Sec. IV G: mu0 H_E = 15.9 T and mu0 H_A = 1 mT give f_AFMR ~ 5.0 GHz (printed)."""
    (BE, BA, f_printed, tol), = read_golden("afm_sec4g.txt")
    Ms = 2e5
    K = BA * Ms / 2
    p = W.make_problem(1, 1, 1, 5e-9, W.full_mask(1, 1, 1), nsub=2, Ms=Ms, alpha=0.0, Ku=K,
                       B0=(0, 0, 0), BE=BE)
    ev = spectrum(p)
    f = np.abs(ev.imag).max() / TP / 1e9
    assert abs(f - f_printed) < tol


# ------------------------------------------------------------------------------------------
# cavity coupling: polariton branches, dissipative coupling, dark mode
# ------------------------------------------------------------------------------------------

def kittel_cavity_matrix(wm, alpha, modes):
    """Linearised Kittel-mode + cavity equations derived by hand from Eqs. (1), (2), (13) and
    the LLG with a transverse field B_x = sum_n (2/gamma) Re[g~_n a_n]:
        dm-/dt = -(alpha + i) gamma' (B0 m- - B_x),   gamma' = gamma/(1+alpha^2)
        da_n/dt = (-i w_n - kappa_n) a_n + i g~_n m-
    in the variables (m-, conj m-, a_1, conj a_1, ...)."""
    N = len(modes)
    n = 2 + 2 * N
    M = np.zeros((n, n), complex)
    gp_B0 = wm  # gamma' B0 with the caller's convention
    cm = -(alpha + 1j) * gp_B0
    M[0, 0] = cm
    M[1, 1] = np.conj(cm)
    for j, (w, k, gt) in enumerate(modes):
        ia, ib = 2 + 2 * j, 3 + 2 * j
        # B_x = (1/gamma)(g~ a + conj(g~) conj(a)); gamma' / gamma = 1/(1+alpha^2)
        fac = (alpha + 1j) / (1 + alpha ** 2)
        M[0, ia] += fac * gt
        M[0, ib] += fac * np.conj(gt)
        M[1, ia] += np.conj(fac) * gt
        M[1, ib] += np.conj(fac) * np.conj(gt)
        M[ia, ia] = -1j * w - k
        M[ib, ib] = 1j * w - k
        M[ia, 0] = 1j * gt
        M[ib, 1] = np.conj(1j * gt)
    return M


@pytest.mark.parametrize("gt_MHz", [50.0, 50.0 + 50.0j, -50.0j])
def test_coupled_kittel_cavity_exact_linearisation(gt_MHz):
    """The oracle's linearised spectrum contains exactly the eigenvalues of the hand-derived
    Kittel + cavity system (coherent, mixed and purely dissipative g~, Eq. (19))."""
    p = W.single_sphere()
    gt = TP * 1e6 * complex(gt_MHz)
    p = p.replace(g_re=np.array([gt.real]), g_im=np.array([gt.imag]))
    ev = spectrum(p)
    wm = G * p.B0[2] / (1 + p.alpha ** 2)
    M = kittel_cavity_matrix(wm, p.alpha, [(p.omega[0], p.kappa[0], gt)])
    for lam in np.linalg.eigvals(M):
        assert abs(nearest(ev, lam) - lam) < 1e-8 * abs(lam)


def test_anticrossing_branches_match_eq6():
    """At resonance with kappa = gamma_m the branches are (w_c + w_m)/2 +- g (Eq. (6)/(7)) up to
    the small counter-rotating shift; sweeping B0 follows Eq. (6) across the anticrossing."""
    p = W.single_sphere()
    wc, g = p.omega[0], p.g_re[0]
    for B0 in np.linspace(0.170, 0.187, 5):
        q = p.replace(B0=np.array([0, 0, B0]))
        ev = spectrum(q)
        wm = G * B0
        for sgn in (+1, -1):
            w = 0.5 * (wc + wm) + sgn * math.sqrt(g * g + (0.5 * (wc - wm)) ** 2)
            lam = nearest(ev, -1j * w)
            assert abs(-lam.imag - w) < TP * 0.1e6       # within 0.1 MHz of Eq. (6)


def test_level_attraction_eq20():
    """Pure dissipative coupling g~ = -i g_d at resonance with kappa = gamma_m: real parts
    coalesce and imaginary parts split by 2 g_d (Eq. (20), Sec. IV H)."""
    p = W.single_sphere()
    gd = TP * 50e6
    p = p.replace(g_re=np.array([0.0]), g_im=np.array([-gd]))
    ev = spectrum(p)
    near = ev[np.abs(np.abs(ev.imag) - p.omega[0]) < TP * 0.3e9]
    near = near[near.imag < 0]
    assert len(near) == 2
    assert abs(near[0].imag - near[1].imag) < TP * 0.1e6
    assert abs(abs(near[0].real - near[1].real) - 2 * gd) < TP * 0.1e6


def test_dark_mode_exact():
    """Two degenerate cavities, a(0) = eps (g2, -g1), m = z: the feedback field
    g1 Re a1 + g2 Re a2 vanishes identically, so m stays on z and each a_n decays as
    exp(-(i w + kappa) t) (the dark state of Eq. (14), Sec. II F)."""
    g1, g2 = TP * 40e6, TP * 70e6
    w, k = TP * 5e9, TP * 3e6
    eps = 1e-2 / math.hypot(g1, g2)
    p = W.make_problem(4, 4, 4, 5e-9, W.sphere_mask(4, 4, 4), B0=(0, 0, w / G),
                       Nd=(1 / 3, 1 / 3, 1 / 3), omega=[w, w], kappa=[k, k], g_re=[g1, g2],
                       g_im=[0, 0], m0=W.tilted_state(1, 4, 4, 4, 0.0, 0.0),
                       a0=np.array([eps * g2, -eps * g1], complex), rtol=1e-8)
    it = O.Integrator(O.OracleProblem(p))
    T = 1e-9
    rc, _ = it.run(T)
    assert rc == 0
    st = it.state()
    m = st["m"].reshape(3, -1)[:, p.mask.reshape(-1) > 0]
    assert np.abs(m[:2]).max() < 1e-12
    want = np.array([eps * g2, -eps * g1]) * np.exp(-(1j * w + k) * T)
    assert np.abs(st["a"] - want).max() < 1e-7 * eps * g2
    # the 3x3 eigenvector at w with no magnon weight is (g2, -g1) (Eq. (14))
    ev_m = kittel_cavity_matrix(w, p.alpha, [(w, k, g1), (w, k, g2)])
    lam, V = np.linalg.eig(ev_m)
    i = np.argmin(np.abs(lam - (-1j * w - k)))
    v = V[:, i]
    assert abs(v[0]) < 1e-12 and abs(v[1]) < 1e-12
    ratio = v[2] / v[4]
    assert abs(ratio - (-g2 / g1)) < 1e-9


def test_cooperativity_golden():
    """With the paper's YIG damping alpha = 3e-4 the oracle's Kittel decay rate gamma_m gives
    the cooperativities printed in Sec. IV C (Eq. (8))."""
    p = W.make_problem(1, 1, 1, 10e-9, W.full_mask(1, 1, 1), alpha=3e-4,
                       B0=(0, 0, TP * 5e9 / G))
    ev = spectrum(p, m=np.array([0, 0, 1.0]))
    gm = -ev[np.argmax(np.abs(ev))].real
    for g, k, C_printed, rel in read_golden("cooperativity_sec4c.txt"):
        C = (TP * g * 1e6) ** 2 / (TP * k * 1e6 * gm)
        assert abs(C - C_printed) <= rel * C_printed + 0.5 * 10 ** math.floor(math.log10(C_printed) - 1)


# ------------------------------------------------------------------------------------------
# overlaps: selection rule and the printed values
# ------------------------------------------------------------------------------------------

def test_overlap_golden_8x8x1():
    """<u> of cos(n pi x / L) on the paper's full 8 x 8 x 1 grid: 1.00, 0.00, 0.00 (Sec. IV D)."""
    rows = read_golden("overlaps_8x8x1.txt")
    orders = [int(r[0]) for r in rows]
    p = W.make_problem(8, 8, 1, 10e-9, W.full_mask(8, 8, 1), omega=[1.0] * 3, kappa=[0] * 3,
                       g_re=[0] * 3, g_im=[0] * 3, u=W.cos_profiles(orders, 8, 8, 1).astype(float))
    op = O.OracleProblem(p)
    m = np.zeros((3, 1, 8, 8))
    m[0] = 1.0                                       # uniform in-plane m: m- = 1
    got = O.overlap(op, m.reshape(-1))
    for (n, printed), v in zip(rows, got):
        assert round(abs(v), 2) == printed
        assert abs(v.imag) < 1e-15


def test_overlap_selection_rule_sphere():
    """Centred sphere: odd-n cos profiles have <u_n m-> = 0 for uniform m by symmetry, the
    uniform profile returns m- itself (Eq. (10)-(11), (18))."""
    n = 12
    orders = [0, 1, 2, 3]
    p = W.make_problem(n, n, n, 5e-9, W.sphere_mask(n, n, n), omega=[1.0] * 4, kappa=[0] * 4,
                       g_re=[0] * 4, g_im=[0] * 4, u=W.cos_profiles(orders, n, n, n).astype(float))
    op = O.OracleProblem(p)
    m = W.tilted_state(1, n, n, n, 20.0, 0.7) * p.mask
    got = O.overlap(op, m.reshape(-1))
    mminus = math.sin(math.radians(20)) * np.exp(-0.7j)
    assert abs(got[0] - mminus) < 1e-14
    assert abs(got[1]) < 1e-15 and abs(got[3]) < 1e-15
    assert abs(got[2]) > 1e-3                     # even n: no selection rule on a sphere


# ------------------------------------------------------------------------------------------
# time integration: Rabi period, error estimator order, library cross-check
# ------------------------------------------------------------------------------------------

def test_vacuum_rabi_period():
    """At resonance with a(0) = 0.01 and m = z, |a|^2 oscillates with period pi/g (Sec. II A,
    IV B; Fig. 3)."""
    p = W.single_sphere(T=16e-9)
    p = p.replace(g_re=np.array([TP * 100e6]), m0=W.tilted_state(1, 8, 8, 8, 0.0, 0.0),
                  a0=np.array([0.01 + 0j]))
    it = O.Integrator(O.OracleProblem(p))
    rc, log = it.run(p.T, log_cap=200000)
    assert rc == 0
    v = log.view()
    t, a2 = v["t"][v["accepted"]], np.abs(v["a"][v["accepted"], 0]) ** 2
    # minima of |a|^2 (energy fully in the magnet): parabolic refinement of discrete minima
    idx = [i for i in range(1, len(a2) - 1) if a2[i] < a2[i - 1] and a2[i] <= a2[i + 1]
           and a2[i] < 0.2 * a2.max()]
    tm = []
    for i in idx:
        y0, y1, y2 = a2[i - 1], a2[i], a2[i + 1]
        x0, x1, x2 = t[i - 1], t[i], t[i + 1]
        A = np.polyfit([x0, x1, x2], [y0, y1, y2], 2)
        tm.append(-A[1] / (2 * A[0]))
    periods = np.diff(tm)
    TR = math.pi / p.g_re[0]
    assert len(periods) >= 2
    assert np.abs(periods / TR - 1).max() < 2e-3


def test_error_estimate_is_fifth_order():
    """The embedded error estimate of one step scales as h^5 (difference of the 5th- and
    4th-order solutions), checked on a precessing, damped macrospin."""
    p = W.make_problem(1, 1, 1, 5e-9, W.full_mask(1, 1, 1), alpha=0.02, B0=(0, 0, 0.2),
                       m0=W.tilted_state(1, 1, 1, 1, 40.0, 0.0))
    errs = []
    for h in (2e-12, 1e-12):
        it = O.Integrator(O.OracleProblem(p))
        rc, log = it.replay([h])
        errs.append(log.view()["err"][0])
    assert abs(math.log2(errs[0] / errs[1]) - 5.0) < 0.15


def test_dp_steps_match_scipy_dop853():
    """Fixed-step Dormand-Prince replay of a small coupled problem converges to scipy's DOP853
    solution (a different integrator on the same right-hand side) at 5th order."""
    from scipy.integrate import solve_ivp
    p = W.make_problem(3, 3, 2, 20e-9, W.full_mask(3, 3, 2), alpha=0.01, Ku=-600.0,
                       B0=(0.01, 0, 0.18), Nd=(0.1, 0.2, 0.7), omega=[TP * 5e9, TP * 5.2e9],
                       kappa=[TP * 5e6, TP * 8e6], g_re=[TP * 60e6, TP * 30e6],
                       g_im=[0, TP * 10e6], u=np.random.default_rng(3).uniform(-1, 1, (2, 2, 3, 3)),
                       a0=np.array([0.004 + 0.001j, -0.002j]))
    p = p.replace(m0=W.random_state(1, 3, 3, 2, seed=5, spread=0.05))
    op = O.OracleProblem(p)
    T = 80e-12
    y0 = np.concatenate([op.m0(), op.a0()])
    nm = len(op.m0())

    def f(t, y):
        dm, da, _ = O.rhs(op, y[:nm], y[nm:])
        return np.concatenate([dm, da])
    ref = solve_ivp(f, (0, T), y0, method="DOP853", rtol=1e-13, atol=1e-15).y[:, -1]
    errs = []
    for nstep in (100, 200, 400):
        it = O.Integrator(op)
        rc, _ = it.replay(np.full(nstep, T / nstep), log=False)
        assert rc == 0
        st = it.state()
        errs.append(max(np.abs(st["m"] - ref[:nm]).max(),
                        np.abs(O.pack_a(st["a"]) - ref[nm:]).max() / np.abs(ref[nm:]).max()))
    assert errs[-1] < 1e-10
    for e1, e2 in zip(errs, errs[1:]):
        assert 4.7 < math.log2(e1 / e2) < 5.6
