"""Seeded synthetic inputs for the coupled LLG + N-cavity-mode integrator.

This module only builds inputs: grids, masks, material constants, mode parameters, mode
profiles u_n(r) and initial states.  It holds none of the integrator's arithmetic, so both the
CUDA path and the FP64 CPU oracle can be fed from it without sharing any computation.

Every generator is deterministic for a given seed.  The material and mode numbers follow the
five workloads the project is measured on (all SI units, frequencies in rad/s, fields in T):

* ``single_sphere``  8x8x8 grid, 5 nm cells, spherical mask, YIG-like film parameters, one
  uniform mode at 5 GHz with g/2pi = 50 MHz, kappa/2pi = 5 MHz (the single-mode Rabi /
  anticrossing set-up of Sec. IV A-B, Eq. (1)-(5)).
* ``multimode_sphere`` 128x128x64 grid, 64-cell-diameter sphere, K_u = -610 J/m^3 along z,
  four standing-wave modes u_n = cos(n pi x / L_x), n = 0..3 (Eq. (11)), at 4.8/5.0/5.2/5.4 GHz.
* ``afm_film``  256x256x16 two-sublattice film, 2 nm cells, B_E = 50 T, K = 5e4 J/m^3, two
  modes near the lower AFMR branch (Eq. (15)-(16)); mode 2 has complex coupling (Eq. (19)-(20)).
* ``batch_sweep``  512 spheres of random size 24^3..96^3 with B0 swept across the anticrossing
  and cooperativities C = g^2/(kappa gamma_m) in [0.1, 50] (Eq. (8)).
* ``adjoint_sphere`` 64^3 sphere, 10 nm cells, three modes with random Fourier profiles.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

GAMMA = 1.76e11          # gyromagnetic ratio used throughout the paper, rad/(s T)
TWO_PI = 2.0 * math.pi
MU0 = 4.0e-7 * math.pi   # vacuum permeability (classical value), T m / A


@dataclasses.dataclass
class Problem:
    """One integration problem: magnet on a box grid + N cavity modes + solver settings.

    Arrays use the dense box layout, x fastest: index = x + nx*(y + ny*z).
    """
    nx: int
    ny: int
    nz: int
    cx: float
    cy: float
    cz: float
    nsub: int                      # 1 = ferromagnet, 2 = two-sublattice antiferromagnet
    mask: np.ndarray               # uint8 (nz, ny, nx); 1 = magnetic cell
    Ms: float                      # saturation magnetisation per sublattice, A/m
    Aex: float                     # intra-sublattice exchange stiffness, J/m
    alpha: float                   # Gilbert damping
    gamma: float                   # rad/(s T)
    Ku: float                      # uniaxial anisotropy constant, J/m^3
    ku_axis: np.ndarray            # unit vector (3,)
    B0: np.ndarray                 # static field (3,), T
    Ndemag: np.ndarray             # diagonal demag factors (3,)
    BE: float                      # inter-sublattice exchange field, T (AFM only)
    omega: np.ndarray              # (N,) cavity frequencies, rad/s
    kappa: np.ndarray              # (N,) cavity amplitude decay rates, rad/s
    g_re: np.ndarray               # (N,) real part of the complex coupling g~_n, rad/s
    g_im: np.ndarray               # (N,) imaginary part of g~_n, rad/s
    u: Optional[np.ndarray]        # (N, nz, ny, nx) mode profiles, or None = all ones
    m0: np.ndarray                 # (nsub, 3, nz, ny, nx) initial unit magnetisation
    a0: np.ndarray                 # (N,) complex initial cavity amplitudes
    T: float = 1e-9                # end time, s
    rtol: float = 1e-6
    a_ref: float = 1e-3            # amplitude floor of the cavity error scale
    dt0: float = 1e-13
    dt_min: float = 1e-18
    dt_max: float = 1e-11
    name: str = ""
    # external drive eta_n(t) = drive_n exp(-(t - drive_t0)^2 / (2 drive_sigma^2)) on da_n/dt
    drive: Optional[np.ndarray] = None   # (N,) complex amplitudes [1/s], or None
    drive_t0: float = 0.1e-9
    drive_sigma: float = 20e-12
    # nonreciprocal coupling: backward (cavity-to-magnon) coefficients of the feedback field,
    # None = reciprocal (the forward g~); self-Kerr coefficients K_n [rad/s per |a|^2] or None
    g_back: Optional[np.ndarray] = None
    kerr: Optional[np.ndarray] = None
    # degenerate parametric pump -i P_n e^{-i wp_n t} conj(a_n) on da_n/dt: complex P_n [rad/s]
    # and the pump frequencies wp_n [rad/s]; None = no pump
    pump: Optional[np.ndarray] = None
    pump_omega: Optional[np.ndarray] = None
    # full magnetostatic demag (cell-pair tensor convolution) instead of the diagonal factors
    full_demag: bool = False

    @property
    def nmodes(self) -> int:
        return int(len(self.omega))

    @property
    def nbox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def ncells(self) -> int:
        return int(self.mask.sum())

    def mask_flat(self) -> np.ndarray:
        return np.ascontiguousarray(self.mask.reshape(-1).astype(np.uint8))

    def m0_flat(self) -> np.ndarray:
        return np.ascontiguousarray(self.m0.reshape(self.nsub, 3, -1))

    def u_flat(self) -> Optional[np.ndarray]:
        if self.u is None:
            return None
        return np.ascontiguousarray(self.u.reshape(self.nmodes, -1))

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------------------------

def sphere_mask(nx: int, ny: int, nz: int, diameter: Optional[float] = None) -> np.ndarray:
    """Cells whose centre lies within radius d/2 of the box centre; d = min(nx, ny, nz) cells."""
    d = float(min(nx, ny, nz)) if diameter is None else float(diameter)
    r2 = (d / 2.0) ** 2
    z, y, x = np.meshgrid(np.arange(nz) + 0.5 - nz / 2.0, np.arange(ny) + 0.5 - ny / 2.0,
                          np.arange(nx) + 0.5 - nx / 2.0, indexing="ij")
    return (x * x + y * y + z * z <= r2 + 1e-9).astype(np.uint8)


def full_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    return np.ones((nz, ny, nx), np.uint8)


def random_mask(nx: int, ny: int, nz: int, fill: float, seed: int) -> np.ndarray:
    """Irregular mask with holes and several x-runs per row (exercises the general layout)."""
    rng = np.random.default_rng(seed)
    return (rng.random((nz, ny, nx)) < fill).astype(np.uint8)


def cos_profiles(orders: List[int], nx: int, ny: int, nz: int) -> np.ndarray:
    """Standing-wave profiles u_n = cos(n pi x / L_x) (Eq. (11)); x = cell-centre coordinate
    measured from the lower box edge, so odd n are antisymmetric about the box centre."""
    x = (np.arange(nx) + 0.5) / nx
    out = np.empty((len(orders), nz, ny, nx), np.float32)
    for i, n in enumerate(orders):
        out[i] = np.cos(n * math.pi * x)[None, None, :].astype(np.float32)
    return out


def fourier_profiles(nmodes: int, nx: int, ny: int, nz: int, seed: int,
                     nterms: int = 8) -> np.ndarray:
    """Random smooth profiles: sum of `nterms` plane waves cos(k.r + phi) with |k| <= 4 pi / L,
    scaled to max |u| = 1 (the learnable-profile initialisation)."""
    rng = np.random.default_rng(seed)
    L = float(max(nx, ny, nz))
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    out = np.empty((nmodes, nz, ny, nx), np.float32)
    for n in range(nmodes):
        acc = np.zeros((nz, ny, nx))
        for _ in range(nterms):
            k = rng.normal(size=3)
            k *= rng.uniform(0.0, 4.0 * math.pi / L) / max(np.linalg.norm(k), 1e-12)
            phi = rng.uniform(0.0, TWO_PI)
            acc += np.cos(k[0] * x + k[1] * y + k[2] * z + phi)
        out[n] = (acc / np.abs(acc).max()).astype(np.float32)
    return out


def tilted_state(nsub: int, nx: int, ny: int, nz: int, theta_deg: float, phi: float,
                 afm: bool = False) -> np.ndarray:
    """Uniform magnetisation tilted by theta from +z at azimuth phi.  For afm=True sublattice 1
    is tilted and sublattice 2 points along -z."""
    th = math.radians(theta_deg)
    m = np.zeros((nsub, 3, nz, ny, nx))
    m[0, 0] = math.sin(th) * math.cos(phi)
    m[0, 1] = math.sin(th) * math.sin(phi)
    m[0, 2] = math.cos(th)
    if nsub == 2:
        if afm:
            m[1, 2] = -1.0
        else:
            m[1] = m[0]
    return m


def _modes(omega, kappa, g_re, g_im):
    return (np.asarray(omega, float), np.asarray(kappa, float), np.asarray(g_re, float),
            np.asarray(g_im, float))


def make_problem(nx, ny, nz, c, mask, *, nsub=1, Ms=1.4e5, Aex=3.7e-12, alpha=1e-3,
                 gamma=GAMMA, Ku=0.0, ku_axis=(0, 0, 1), B0=(0, 0, 0.1785), Nd=(0, 0, 0),
                 BE=0.0, omega=(), kappa=(), g_re=(), g_im=(), u=None, m0=None, a0=None,
                 **solver) -> Problem:
    omega, kappa, g_re, g_im = _modes(omega, kappa, g_re, g_im)
    n = len(omega)
    if m0 is None:
        m0 = tilted_state(nsub, nx, ny, nz, 1.0, 0.0, afm=(nsub == 2))
    if a0 is None:
        a0 = np.zeros(n, complex)
    cx, cy, cz = (c, c, c) if np.isscalar(c) else c
    return Problem(nx=nx, ny=ny, nz=nz, cx=cx, cy=cy, cz=cz, nsub=nsub,
                   mask=np.asarray(mask, np.uint8), Ms=Ms, Aex=Aex, alpha=alpha, gamma=gamma,
                   Ku=Ku, ku_axis=np.asarray(ku_axis, float), B0=np.asarray(B0, float),
                   Ndemag=np.asarray(Nd, float), BE=BE, omega=omega, kappa=kappa, g_re=g_re,
                   g_im=g_im, u=u, m0=np.asarray(m0, float), a0=np.asarray(a0, complex),
                   **solver)


# ----------------------------------------------------------------------------------------------
# the five measured workloads
# ----------------------------------------------------------------------------------------------

def single_sphere(T=20e-9) -> Problem:
    """8^3 grid, 5 nm cells, sphere; one uniform mode; B0 so that gamma*B0 = 2 pi 5 GHz."""
    n = 8
    B0 = TWO_PI * 5e9 / GAMMA
    return make_problem(n, n, n, 5e-9, sphere_mask(n, n, n), Ms=1.4e5, Aex=3.7e-12,
                        alpha=1e-3, B0=(0, 0, B0), Nd=(1 / 3, 1 / 3, 1 / 3),
                        omega=[TWO_PI * 5e9], kappa=[TWO_PI * 5e6], g_re=[TWO_PI * 50e6],
                        g_im=[0.0], m0=tilted_state(1, n, n, n, 1.0, 0.0), T=T,
                        name="single_sphere_8^3")


def multimode_sphere(T=10e-9, seed=2603, nx=128, ny=128, nz=64) -> Problem:
    """128x128x64, sphere of 64-cell diameter, K_u = -610 J/m^3 (z), four cos(n pi x/L_x) modes.
    B0 is chosen so that the Kittel frequency including the anisotropy field is 5.0 GHz."""
    rng = np.random.default_rng(seed)
    Ku, Ms = -610.0, 1.4e5
    B0 = TWO_PI * 5e9 / GAMMA - 2.0 * Ku / Ms
    g = TWO_PI * rng.uniform(20e6, 80e6, size=4)
    phi = rng.uniform(0.0, TWO_PI)
    f = np.array([4.8e9, 5.0e9, 5.2e9, 5.4e9])
    p = make_problem(nx, ny, nz, 5e-9, sphere_mask(nx, ny, nz), Ms=Ms, Aex=3.7e-12,
                     alpha=1e-3, Ku=Ku, B0=(0, 0, B0), Nd=(1 / 3, 1 / 3, 1 / 3),
                     omega=TWO_PI * f, kappa=np.full(4, TWO_PI * 2e6), g_re=g,
                        g_im=np.zeros(4), u=cos_profiles([0, 1, 2, 3], nx, ny, nz),
                        m0=tilted_state(1, nx, ny, nz, 1.0, phi), T=T,
                        name="multimode_sphere_128x128x64")
    return p.replace(dt_max=stable_dt_max(p))


def afm_params():
    """AFM constants: B_A = 2K/Ms, f_AFMR = gamma sqrt(2 B_E B_A + B_A^2) / 2pi (Eq. (15)), lower
    branch f_- = f_AFMR - gamma B / 2pi at B = 1 T (Eq. (16))."""
    Ms, K, BE, B = 4e5, 5e4, 50.0, 1.0
    BA = 2 * K / Ms
    w_afmr = GAMMA * math.sqrt(2 * BE * BA + BA * BA)
    w_minus = w_afmr - GAMMA * B
    return dict(Ms=Ms, K=K, BE=BE, B=B, BA=BA, w_afmr=w_afmr, w_minus=w_minus)


def afm_film(T=5e-9, nx=256, ny=256, nz=16) -> Problem:
    p = afm_params()
    wm = p["w_minus"]
    omega = [wm - TWO_PI * 60e6, wm + TWO_PI * 60e6]
    return make_problem(nx, ny, nz, 2e-9, full_mask(nx, ny, nz), nsub=2, Ms=p["Ms"],
                        Aex=5e-12, alpha=2e-3, Ku=p["K"], B0=(0, 0, p["B"]), Nd=(0, 0, 1),
                        BE=p["BE"], omega=omega, kappa=[TWO_PI * 2e6] * 2,
                        g_re=[TWO_PI * 30e6] * 2, g_im=[0.0, TWO_PI * 30e6],
                        m0=tilted_state(2, nx, ny, nz, 1.0, 0.0, afm=True), T=T,
                        name="afm_film_256x256x16")


def batch_sweep(n_inst=512, seed=3706, T=30e-9, nmin=24, nmax=96) -> List[Problem]:
    """Independent spheres of random size; omega_m/2pi swept linearly 4.6 -> 5.4 GHz over the
    index; 1-3 modes at 5.0, 4.85, 5.15 GHz; log C ~ U[log 0.1, log 50], kappa/2pi ~ U[1, 10] MHz,
    g = sqrt(C kappa gamma_m) redrawn until g/2pi lies in [5, 80] MHz."""
    rng = np.random.default_rng(seed)
    alpha = 1e-3
    out = []
    for i in range(n_inst):
        n = int(rng.integers(nmin, nmax + 1))
        fm = 4.6e9 + 0.8e9 * (i / max(n_inst - 1, 1))
        B0 = TWO_PI * fm / GAMMA
        nm = int(rng.integers(1, 4))
        fc = [5.0e9, 4.85e9, 5.15e9][:nm]
        gm = alpha * TWO_PI * fm
        g, kap = [], []
        for _ in range(nm):
            while True:
                C = math.exp(rng.uniform(math.log(0.1), math.log(50.0)))
                k = TWO_PI * rng.uniform(1e6, 10e6)
                gg = math.sqrt(C * k * gm)
                if TWO_PI * 5e6 <= gg <= TWO_PI * 80e6:
                    break
            g.append(gg)
            kap.append(k)
        out.append(make_problem(n, n, n, 5e-9, sphere_mask(n, n, n), alpha=alpha,
                                B0=(0, 0, B0), Nd=(1 / 3, 1 / 3, 1 / 3),
                                omega=TWO_PI * np.array(fc), kappa=kap, g_re=g,
                                g_im=np.zeros(nm), m0=tilted_state(1, n, n, n, 1.0, 0.0),
                                T=T, name=f"batch_{i}_n{n}"))
    return out


def adjoint_sphere(T=20e-9, n=64, seed=42) -> Problem:
    """64^3 sphere, 10 nm cells; cavities at 4.95 / 5.20 / 5.05 GHz, g/2pi = 50 MHz; a_1(0) =
    0.01, m = +z; profiles are random Fourier fields."""
    B0 = TWO_PI * 5e9 / GAMMA
    m0 = tilted_state(1, n, n, n, 0.0, 0.0)
    p = make_problem(n, n, n, 10e-9, sphere_mask(n, n, n), alpha=1e-3, B0=(0, 0, B0),
                     Nd=(1 / 3, 1 / 3, 1 / 3), omega=TWO_PI * np.array([4.95e9, 5.20e9, 5.05e9]),
                     kappa=[TWO_PI * 1e6] * 3, g_re=[TWO_PI * 50e6] * 3, g_im=[0.0] * 3,
                     u=fourier_profiles(3, n, n, n, seed), m0=m0,
                     a0=np.array([0.01, 0, 0], complex), T=T, name="adjoint_sphere_64^3")
    return p.replace(dt_max=stable_dt_max(p))


def spectral_radius(p: Problem) -> float:
    """Upper bound (rad/s) on the linear spin-wave frequencies of the LLG right-hand side: the
    exchange Laplacian contributes at most (2A/Ms) sum_d 4/c_d^2; two sublattices add the
    inter-sublattice field (omega <= gamma (B + B_A + lambda + B_E), Eq. (15)-(16))."""
    lam = 2.0 * p.Aex / p.Ms * sum(4.0 / c ** 2 for c in (p.cx, p.cy, p.cz))
    b = (float(np.linalg.norm(p.B0)) + abs(2.0 * p.Ku / p.Ms)
         + MU0 * p.Ms * float(np.max(np.abs(p.Ndemag))) * p.nsub + lam)
    if p.nsub == 2:
        b += abs(p.BE)
    return p.gamma / math.sqrt(1.0 + p.alpha ** 2) * b


def stable_dt_max(p: Problem, y_max: float = 1.2) -> float:
    """Step-size cap keeping every spin wave inside the Dormand-Prince stability region
    (|R(z)| <= 1 up to |z| ~ 1.2 near the imaginary axis for alpha >= 1e-3).  Used whenever
    the drive or the state is spatially non-uniform, so that exchange modes are never amplified
    by accepted steps; exactly uniform problems do not excite them and keep dt_max = 1e-11."""
    return min(p.dt_max, y_max / spectral_radius(p))


def random_state(nsub, nx, ny, nz, seed, spread=0.3, afm=False) -> np.ndarray:
    """Smoothly random unit vectors near +z (or -z on sublattice 2 for afm): small random
    deviations, then normalised.  Used for single-stage parity checks."""
    rng = np.random.default_rng(seed)
    m = rng.normal(scale=spread, size=(nsub, 3, nz, ny, nx))
    m[:, 2] += 1.0
    if afm and nsub == 2:
        m[1, 2] -= 2.0
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    return m
