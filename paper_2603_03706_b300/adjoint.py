"""Differentiable runs of the coupled system for PyTorch: a torch.autograd.Function over the CUDA
integrator (forward: cmx_run with the checkpoint store armed) and its discrete adjoint
(backward: cmx_adjoint).  Only argument marshalling happens here; every step of the forward and
of the reverse sweep runs in libcmx.

The outputs are the cavity amplitudes after every accepted step, a_traj[i, n, (Re, Im)] with
a_traj[0] = a_0, their times, and the final magnetisation; any loss built from them with torch
operations can be differentiated with respect to Re g~_n, Im g~_n, kappa_n, omega_n, alpha, the
per-cell profiles u_n(r), a_0 and m_0.  The accepted step sizes are held fixed in the backward
pass (discrete adjoint of the accepted steps).

Two losses of the kind the paper's multimode experiments call for (Sec. IV C, D) are provided:
``energy_transfer`` (cavity i -> cavity j, |a_j(T)|^2 / |a_i(0)|^2) and ``splitting`` (the
frequency distance of the two strongest complex exponentials in one cavity's trace, from a
linear-prediction fit that torch can differentiate).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import cmx


@dataclasses.dataclass
class RunSpec:
    """Everything about a run that is not differentiated: the Problem supplies geometry,
    material, solver settings and end time; `every` is the checkpoint spacing in accepted
    steps and `max_steps` the largest accepted-step count the run may take."""
    problem: object
    every: int = 200
    max_steps: int = 200000
    log_cap: Optional[int] = None


def _np(x, dtype):
    return np.ascontiguousarray(x.detach().cpu().numpy(), dtype=dtype)


class CoupledRun(torch.autograd.Function):
    """forward(g_re, g_im, kappa, omega, alpha, u, a0, m0, spec) -> (a_traj, t, m_T)

    g_re, g_im, kappa, omega: (N,) float64 [rad/s]; alpha: () float64; u: (N, nz, ny, nx)
    float32 (CPU or CUDA) or None; a0: (N, 2) float64 (Re, Im); m0: (nsub, 3, nz, ny, nx)
    float32.  a_traj: (n+1, N, 2) float64; t: (n+1,) float64 (not differentiable);
    m_T: (nsub, 3, nz, ny, nx) float32.
    """

    @staticmethod
    def forward(ctx, g_re, g_im, kappa, omega, alpha, u, a0, m0, spec: RunSpec):
        p = spec.problem
        a0c = _np(a0, np.float64)
        p = p.replace(g_re=_np(g_re, np.float64), g_im=_np(g_im, np.float64),
                      kappa=_np(kappa, np.float64), omega=_np(omega, np.float64),
                      alpha=float(alpha.detach().cpu()), a0=a0c[:, 0] + 1j * a0c[:, 1],
                      m0=_np(m0, np.float32).astype(np.float64))
        log_cap = spec.log_cap or (2 * spec.max_steps + 64)
        uarg = None if u is None else (u.detach().contiguous() if u.is_cuda
                                       else _np(u, np.float32))
        sim = cmx.Simulation.from_problem(p.replace(u=None), log_cap=log_cap, u=uarg)
        sim.adjoint_record(spec.every, spec.max_steps)
        sim.run(p.T)
        log = sim.get_log()
        acc = log["accepted"]
        N = p.nmodes
        a_steps = log["a"][acc] if N else np.zeros((int(acc.sum()), 0), complex)
        traj = np.concatenate([(a0c[:, 0] + 1j * a0c[:, 1])[None], a_steps])
        t = np.concatenate([[0.0], log["t"][acc]])
        m_T = sim.get_m()
        ctx.sim = sim
        ctx.has_u = u is not None
        ctx.u_meta = (u.dtype, u.device) if u is not None else None
        ctx.m0_meta = (m0.dtype, m0.device)
        a_traj = torch.from_numpy(np.stack([traj.real, traj.imag], -1)).to(torch.float64)
        t_out = torch.from_numpy(t)
        ctx.mark_non_differentiable(t_out)
        return a_traj, t_out, torch.from_numpy(np.asarray(m_T, np.float32)).to(m0.device)

    @staticmethod
    def backward(ctx, g_traj, g_t, g_mT):
        sim = ctx.sim
        la = None if g_traj is None else _np(g_traj, np.float64).reshape(g_traj.shape[0], -1)
        lm = None if g_mT is None else _np(g_mT, np.float32)
        g = sim.adjoint(la, lm, want_u=ctx.has_u, want_m0=True)
        sim.close()
        ctx.sim = None
        f64 = lambda v: torch.as_tensor(np.asarray(v, np.float64))
        d_a0 = torch.as_tensor(np.stack([g["a0"].real, g["a0"].imag], -1))
        d_u = None
        if ctx.has_u:
            d_u = torch.as_tensor(g["u"]).to(dtype=ctx.u_meta[0], device=ctx.u_meta[1])
        d_m0 = torch.as_tensor(g["m0"]).to(dtype=ctx.m0_meta[0], device=ctx.m0_meta[1])
        return (f64(g["g_re"]), f64(g["g_im"]), f64(g["kappa"]), f64(g["omega"]),
                f64(g["alpha"]).reshape(()), d_u, d_a0, d_m0, None)


def run(g_re, g_im, kappa, omega, alpha, u, a0, m0, spec: RunSpec):
    """Differentiable run; see CoupledRun."""
    return CoupledRun.apply(g_re, g_im, kappa, omega, alpha, u, a0, m0, spec)


def parameters_from(problem, device=None, requires_grad=True):
    """Torch leaves holding a Problem's learnable values (for an optimiser)."""
    p = problem
    rg = requires_grad
    t64 = lambda v: torch.tensor(np.asarray(v, np.float64), requires_grad=rg)
    out = dict(g_re=t64(p.g_re), g_im=t64(p.g_im), kappa=t64(p.kappa), omega=t64(p.omega),
               alpha=torch.tensor(float(p.alpha), dtype=torch.float64, requires_grad=rg),
               a0=torch.tensor(np.stack([np.real(p.a0), np.imag(p.a0)], -1), dtype=torch.float64,
                               requires_grad=rg),
               m0=torch.tensor(np.asarray(p.m0, np.float32), requires_grad=False))
    out["u"] = None if p.u is None else torch.tensor(np.asarray(p.u, np.float32),
                                                      device=device, requires_grad=rg)
    return out


def energy_transfer(a_traj: torch.Tensor, i: int, j: int) -> torch.Tensor:
    """|a_j(T)|^2 / |a_i(0)|^2: the fraction of cavity i's initial energy found in cavity j
    at the end of the run."""
    return a_traj[-1, j].pow(2).sum() / a_traj[0, i].pow(2).sum()


def splitting(a_traj: torch.Tensor, t: torch.Tensor, mode: int, n_samples: int = 64,
              t_start: float = 0.0, w_ref: Optional[float] = None) -> torch.Tensor:
    """Frequency distance |w_+ - w_-| (rad/s) of the two polariton branches seen in one cavity's
    trace.  The trace is shifted to base band, y e^{i w_ref t} (w_ref: the mean rotation of the
    trace unless given; the distance does not depend on it), resampled linearly onto a uniform
    grid of n_samples points, and a two-term linear predictor y_{k+2} = c_1 y_{k+1} + c_0 y_k
    is fitted by least squares; the roots z of z^2 - c_1 z - c_0 give the two branches,
    w = w_ref - arg(z) / dt (e^{-i w t} convention).  Base band keeps the two roots well apart
    on the unit circle, where the fit is well conditioned."""
    t = t.to(torch.float64)
    y = torch.complex(a_traj[:, mode, 0], a_traj[:, mode, 1])
    keep = t >= t_start
    t, y = t[keep], y[keep]
    if w_ref is None:
        ph = np.unwrap(np.angle(y.detach().cpu().numpy()))
        w_ref = -(ph[-1] - ph[0]) / float(t[-1] - t[0])
    yb = y * torch.exp(1j * w_ref * t)
    tu = torch.linspace(float(t[0]), float(t[-1]), n_samples, dtype=torch.float64)
    k = torch.clamp(torch.searchsorted(t, tu, right=True) - 1, 0, len(t) - 2)
    w = (tu - t[k]) / (t[k + 1] - t[k])
    yu = yb[k] * (1 - w) + yb[k + 1] * w
    dt = float(tu[1] - tu[0])
    A = torch.stack([yu[1:-1], yu[:-2]], -1)
    b = yu[2:]
    Ah = A.conj().transpose(0, 1)
    c = torch.linalg.solve(Ah @ A, Ah @ b)
    disc = torch.sqrt(c[0] * c[0] + 4 * c[1])
    z1, z2 = (c[0] + disc) / 2, (c[0] - disc) / 2
    return (torch.angle(z1) - torch.angle(z2)).abs() / dt
