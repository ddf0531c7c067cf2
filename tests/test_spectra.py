"""The matrix-pencil estimator recovers known damped exponentials (CPU only)."""
import math

import numpy as np

from paper_2603_03706_b300 import spectra

TP = 2 * math.pi


def test_matrix_pencil_recovers_two_branches():
    dt = 5e-12
    t = np.arange(4000) * dt
    w = TP * np.array([4.95e9, 5.05e9])
    g = TP * np.array([5e6, 4e6])
    c = np.array([0.6 + 0.2j, -0.3 + 0.5j])
    y = (c[None, :] * np.exp(-(g + 1j * w)[None, :] * t[:, None])).sum(1)
    om, ga, amp = spectra.matrix_pencil(y, dt, 2)
    o = np.argsort(om)
    assert np.abs(om[o] - w).max() < TP * 10.0          # 10 Hz
    assert np.abs(ga[o] - g).max() < TP * 10.0
    assert np.allclose(amp[o], c, rtol=1e-6)


def test_polariton_branches_reduce_to_eq6():
    wc, wm, g = TP * 5.0e9, TP * 5.02e9, TP * 50e6
    p, m = spectra.polariton_branches(wc, wm, g)
    r = math.sqrt(g * g + ((wc - wm) / 2) ** 2)
    assert abs(p - ((wc + wm) / 2 + r)) < 1e-6 and abs(m - ((wc + wm) / 2 - r)) < 1e-6
    # equal losses shift both branches by -i kappa only (Eq. (7))
    p2, m2 = spectra.polariton_branches(wc, wm, g, kappa=TP * 5e6, gamma_m=TP * 5e6)
    assert abs(p2 - (p - 1j * TP * 5e6)) < 1e-3 and abs(m2 - (m - 1j * TP * 5e6)) < 1e-3
