"""The dense-box stage path (tensor copies; needs a B300) against the FP64 oracle and against the
per-thread-copy path on the same grids.  Dense boxes are grids magnetic over the whole box
(films, full boxes); their rows are stored back to back and each stage loads a plane's tile, halo
and operands with tensor copies whose out-of-box positions read as zero.

* one stage on boxes with a ragged tail in x, y and z (nx not a multiple of 8 or 32, ny not a
  multiple of the tile height), one and two sublattices, with and without mode profiles, every
  compiled tile height, few and many planes per block;
* 1000 replayed adaptive steps (max|dm| <= 2e-5, |da|/max|a| <= 1e-4, the controller's step
  sizes and error norms against reading C6 and the oracle);
* the same adaptive run with plain copies agrees with the dense path;
* the adjoint's recompute runs on the dense path: gradients against the oracle's adjoint;
* the launch reports the dense path for boxes and not for masked grids.
"""
import math

import numpy as np
import pytest

from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

from gpu_util import TOL_A, TOL_M, f32_profiles, f32_state, masked, replay_compare, sim_for
from test_gpu_adjoint import TOL_G, compare, forward, loss_weights, oracle_grads
from test_gpu_parity import rhs_compare

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


def dense_problem(nsub=1, nmodes=2, shape=(37, 21, 11), seed=0, profiles=True):
    nx, ny, nz = shape
    mask = W.full_mask(nx, ny, nz)
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (nmodes, nz, ny, nx)).astype(np.float32) if (nmodes and profiles) \
        else None
    kw = dict(omega=TP * rng.uniform(4.8e9, 5.2e9, nmodes), kappa=TP * rng.uniform(1e6, 5e6, nmodes),
              g_re=TP * rng.uniform(20e6, 80e6, nmodes), g_im=TP * rng.uniform(-30e6, 30e6, nmodes),
              u=u)
    if nsub == 2:
        p = W.make_problem(nx, ny, nz, 2e-9, mask, nsub=2, Ms=4e5, Aex=5e-12, alpha=2e-3, Ku=5e4,
                           B0=(0, 0, 1.0), Nd=(0, 0, 1), BE=50.0, **kw)
    else:
        p = W.make_problem(nx, ny, nz, 5e-9, mask, Ku=-610.0, ku_axis=(0.6, 0.0, 0.8),
                           B0=(0.01, 0, 0.187), Nd=(0.3, 0.3, 0.4), **kw)
    m = W.random_state(nsub, nx, ny, nz, seed + 1, spread=0.2, afm=(nsub == 2))
    a = (rng.normal(size=nmodes) + 1j * rng.normal(size=nmodes)) * 3e-3
    p = p.replace(m0=m, a0=a)
    return p.replace(dt_max=W.stable_dt_max(p))


TILINGS = [(32, 4, 4), (32, 8, 3), (32, 16, 2), (32, 4, 1), (32, 8, 1), (32, 16, 1), (32, 8, 2, 1)]


@pytest.mark.parametrize("tiling", TILINGS)
@pytest.mark.parametrize("nsub", [1, 2])
def test_rhs_dense_box_ragged(tiling, nsub):
    r = rhs_compare(dense_problem(nsub=nsub, seed=3 + nsub), tiling)
    assert r["err_m"] < 2e-6 and r["outside"] == 0.0, r
    assert r["err_mm"] < 1e-7 and r["err_da"] < 1e-6, r


@pytest.mark.parametrize("shape", [(70, 9, 3), (8, 33, 5), (256, 4, 2), (1, 1, 1), (5, 3, 17)])
def test_rhs_dense_shapes_without_profiles(shape):
    r = rhs_compare(dense_problem(nmodes=3, shape=shape, seed=7, profiles=False))
    assert r["err_m"] < 2e-6 and r["outside"] == 0.0, r
    assert r["err_mm"] < 1e-7 and r["err_da"] < 1e-6, r


def test_dense_path_is_taken_only_for_boxes():
    p = f32_state(dense_problem())
    sim = sim_for(p, log_cap=0, tiling=(32, 8, 4))
    assert sim.get_tiling()["dense"] == 1
    sim.close()
    sim = sim_for(p, log_cap=0, tiling=(32, 8, 4, 0, 1))   # plain copies asked for
    assert sim.get_tiling()["dense"] == 0
    sim.close()
    q = p.replace(mask=W.sphere_mask(p.nx, p.ny, p.nz, 9.0))
    sim = sim_for(f32_state(q), log_cap=0, tiling=(32, 8, 4))
    assert sim.get_tiling()["dense"] == 0
    sim.close()


@pytest.mark.parametrize("nsub,tiling", [(1, (32, 4, 4)), (1, (32, 16, 2)), (2, (32, 8, 3)),
                                         (2, (32, 4, 1))])
def test_replay_dense_1000_steps(nsub, tiling):
    p = dense_problem(nsub=nsub, nmodes=2, seed=20 + nsub)
    if nsub == 1:
        p = p.replace(m0=W.tilted_state(1, p.nx, p.ny, p.nz, 5.0, 0.3))
    else:
        p = p.replace(m0=W.tilted_state(2, p.nx, p.ny, p.nz, 1.0, 0.0, afm=True), u=None)
    p = p.replace(a0=np.array([1e-3, 0j]), T=1e-6)
    p = p.replace(dt_max=W.stable_dt_max(p))
    dm, da, info = replay_compare(p, 1000, tiling=tiling)
    assert info["tiling"]["dense"] == 1
    assert dm <= TOL_M and da <= TOL_A, (dm, da)


def test_dense_and_plain_copies_agree():
    p = f32_state(f32_profiles(dense_problem(nsub=2, nmodes=2, seed=31)))
    p = p.replace(m0=f32_state(p.replace(m0=W.tilted_state(2, p.nx, p.ny, p.nz, 2.0, 0.1,
                                                             afm=True))).m0, T=1e-6)
    out = []
    for t in ((32, 8, 4), (32, 8, 4, 0, 1)):
        sim = sim_for(p, log_cap=256, tiling=t)
        sim.run(p.T, max_attempts=200)
        out.append((sim.get_m(), sim.get_a(), sim.get_log()["dt"]))
        sim.close()
    (m0, a0, d0), (m1, a1, d1) = out
    n = min(len(d0), len(d1))
    assert n > 150 and np.allclose(d0[:n], d1[:n], rtol=1e-5)
    if len(d0) == len(d1):
        assert np.abs(masked(p, m0) - masked(p, m1)).max() <= 1e-5
        assert np.abs(a0 - a1).max() <= 1e-5 * np.abs(a1).max()


def test_dense_adjoint_matches_oracle():
    p = dense_problem(nsub=1, nmodes=2, shape=(20, 12, 6), seed=41)
    p = p.replace(m0=W.tilted_state(1, p.nx, p.ny, p.nz, 3.0, 0.2), T=0.2e-9)
    p = f32_state(f32_profiles(p.replace(dt_max=W.stable_dt_max(p))))
    sim, dts, traj = forward(p, 25, tiling=(32, 8, 2))
    assert sim.get_tiling()["dense"] == 1 and len(dts) > 50
    la, wm = loss_weights(p, traj)
    g = sim.adjoint(la, wm)
    sim.close()
    go = oracle_grads(p, dts, la, wm)
    errs = compare(p, g, go)
    assert all(v <= TOL_G for v in errs.values()), errs


def test_dense_replay_with_cavity_extensions():
    """Drive pulse, nonreciprocal coupling, Kerr term and parametric pump on a dense box: the
    cavity work sits in the controller, shared by both copy paths; this runs it after the dense
    stages (1000 replayed steps against the oracle)."""
    p = dense_problem(nsub=1, nmodes=2, seed=51)
    p = p.replace(m0=W.tilted_state(1, p.nx, p.ny, p.nz, 4.0, 0.1), a0=np.array([2e-3, 1e-3j]),
                  T=1e-6)
    p = p.replace(g_back=TP * np.array([25e6 + 5e6j, 70e6 - 10e6j]),
                  kerr=TP * np.array([4e10, -2e10]),
                  pump=TP * np.array([3e6 + 1e6j, -2e6 + 4e6j]),
                  pump_omega=TP * np.array([10.0e9, 10.3e9]),
                  drive=np.array([4e7 + 1e7j, -2e7j]), drive_t0=20e-12, drive_sigma=10e-12)
    p = p.replace(dt_max=W.stable_dt_max(p))
    sim = sim_for(f32_state(f32_profiles(p)), log_cap=0, tiling=(32, 8, 4))
    assert sim.get_tiling()["dense"] == 1
    sim.close()
    dm, da, info = replay_compare(p, 1000, tiling=(32, 8, 4))
    assert dm <= TOL_M and da <= TOL_A, (dm, da)
