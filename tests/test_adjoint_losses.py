"""Host-side pins of the differentiable losses of the adjoint form (CPU only): the splitting
estimator recovers the branch distance of a known two-tone trace sampled at irregular times, and
torch's gradient of both losses matches central differences."""
import math

import numpy as np
import torch

from paper_2603_03706_b300 import adjoint as AD

TP = 2 * math.pi


def two_tone(n=3000, seed=0, f1=4.95e9, f2=5.05e9, T=20e-9):
    rng = np.random.default_rng(seed)
    t = np.sort(np.concatenate([[0.0, T], rng.uniform(0, T, n - 2)]))
    y = (0.6 * np.exp(-1j * TP * f1 * t) + 0.4 * np.exp(-1j * TP * f2 * t)) * np.exp(-t / 50e-9)
    return t, torch.tensor(np.stack([y.real, y.imag], -1)[:, None, :])


def test_splitting_recovers_two_tone_distance():
    t, tr = two_tone()
    for ns in (32, 64, 128):
        s = float(AD.splitting(tr, torch.tensor(t), 0, n_samples=ns))
        assert abs(s - TP * 100e6) <= 1e-4 * TP * 100e6, (ns, s / TP)


def test_splitting_gradient_matches_central_differences():
    t, tr = two_tone(n=600)
    tr = tr.clone().requires_grad_(True)
    tt = torch.tensor(t)
    AD.splitting(tr, tt, 0, w_ref=TP * 5e9).backward()
    rng = np.random.default_rng(1)
    for _ in range(5):
        i, c = int(rng.integers(1, len(t) - 1)), int(rng.integers(0, 2))
        e = torch.zeros_like(tr)
        e[i, 0, c] = 1e-6
        with torch.no_grad():
            fd = (AD.splitting(tr + e, tt, 0, w_ref=TP * 5e9) -
                  AD.splitting(tr - e, tt, 0, w_ref=TP * 5e9)) / 2e-6
        g = float(tr.grad[i, 0, c])
        assert abs(float(fd) - g) <= 1e-4 * max(abs(g), 1e3), (i, c, float(fd), g)


def test_energy_transfer_value_and_gradient():
    a = torch.tensor([[[0.01, 0.002], [0.0, 0.0]], [[0.005, 0.0], [0.003, -0.004]]],
                     dtype=torch.float64, requires_grad=True)
    L = AD.energy_transfer(a, 0, 1)
    Lv = L.item()
    assert abs(Lv - (0.003 ** 2 + 0.004 ** 2) / (0.01 ** 2 + 0.002 ** 2)) < 1e-15
    L.backward()
    e0 = 0.01 ** 2 + 0.002 ** 2
    assert np.allclose(a.grad[1, 1].numpy(), 2 * np.array([0.003, -0.004]) / e0)
    assert np.allclose(a.grad[0, 0].numpy(), -2 * Lv / e0 * np.array([0.01, 0.002]))
