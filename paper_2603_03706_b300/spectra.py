"""Spectral analysis of cavity and magnetisation traces (host side, NumPy).

The paper extracts polariton frequencies from FFT peaks of a(t) and m^-(t) (Sec. IV A, C); a
20 ns trace only resolves 50 MHz bins that way.  Here a sum of damped complex exponentials
    y(t_k) = sum_i c_i exp(lambda_i t_k),   lambda_i = -Gamma_i - i omega_i
is fitted with the matrix-pencil method (Hua & Sarkar, IEEE Trans. ASSP 38, 814 (1990)), which
locates each branch to well below the bin width.  Frequencies follow the e^{-i omega t}
convention of Eq. (1)-(2): a cavity mode at omega_c shows up as omega_i = +omega_c.
"""
from __future__ import annotations

import numpy as np


def matrix_pencil(y: np.ndarray, dt: float, order: int, pencil: int | None = None):
    """Fit `order` damped exponentials to uniform samples y (complex) with spacing dt.

    Returns (omega [rad/s], gamma [1/s], amplitude [complex]) sorted by |amplitude|, largest
    first.
    """
    y = np.asarray(y, complex).reshape(-1)
    L = len(y)
    P = pencil if pencil is not None else L // 3
    if not (order <= P <= L - order):
        raise ValueError("pencil parameter out of range")
    # Hankel data matrix, (L - P) x (P + 1)
    idx = np.arange(L - P)[:, None] + np.arange(P + 1)[None, :]
    Y = y[idx]
    _, _, Vh = np.linalg.svd(Y, full_matrices=False)
    V = Vh[:order].T                             # (P+1) x order: rows of Vh span the signal
    V1, V2 = V[:-1], V[1:]
    z = np.linalg.eigvals(np.linalg.pinv(V1) @ V2)
    lam = np.log(z) / dt
    omega = -lam.imag
    gamma = -lam.real
    # amplitudes by least squares on the Vandermonde system
    t = np.arange(L) * dt
    A = np.exp(np.outer(t, lam))
    c, *_ = np.linalg.lstsq(A, y, rcond=None)
    o = np.argsort(-np.abs(c))
    return omega[o], gamma[o], c[o]


def resample(t: np.ndarray, y: np.ndarray, dt: float, t0: float | None = None,
             t1: float | None = None):
    """Linear resampling of an irregular trace onto a uniform grid."""
    t0 = t[0] if t0 is None else t0
    t1 = t[-1] if t1 is None else t1
    n = int(np.floor((t1 - t0) / dt)) + 1
    tu = t0 + dt * np.arange(n)
    return tu, np.interp(tu, t, y.real) + 1j * np.interp(tu, t, y.imag)


def polariton_branches(wc: float, wm: float, g: complex, kappa: float = 0.0,
                       gamma_m: float = 0.0):
    """Complex branches of Eq. (7)/(20): (w~c + w~m)/2 +- sqrt(g~^2 + ((w~c - w~m)/2)^2) with
    w~c = wc - i kappa, w~m = wm - i gamma_m.  Returns (omega_plus, omega_minus) complex."""
    wct, wmt = wc - 1j * kappa, wm - 1j * gamma_m
    r = np.sqrt(g * g + ((wct - wmt) / 2) ** 2)
    return (wct + wmt) / 2 + r, (wct + wmt) / 2 - r
