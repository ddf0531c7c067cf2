"""Full magnetostatic demag on the device (FFT convolution) against the oracle's direct sum of
the Newell cell-pair tensor (needs a B300).

* single right-hand sides with full demag: a sphere, a box with holes and ragged edges in every
  direction, a thin film, two sublattices;
* 1000 adaptive steps replayed by the oracle (error norms and step sizes checked);
* switching back to the diagonal factors restores the plain path; the modes that do not take
  full demag reject it.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

from gpu_util import TOL_A, TOL_M, f32_profiles, f32_state, masked, replay_compare, sim_for

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


def rhs_compare(p):
    p = f32_state(f32_profiles(p))
    sim = sim_for(p, log_cap=0)
    dm_g, da_g, mm_g = sim.eval_rhs(np.asarray(p.m0, np.float32), p.a0)
    sim.close()
    op = O.OracleProblem(p)
    dm_o, da_o, mm_o = O.rhs(op, op.m0(), O.pack_a(p.a0))
    dm_o = dm_o.reshape(p.nsub, 3, p.nz, p.ny, p.nx)
    scale = np.abs(masked(p, dm_o)).max()
    res = dict(err_m=np.abs(masked(p, dm_g) - masked(p, dm_o)).max() / scale)
    if p.nmodes:
        res["err_da"] = np.abs(da_g - O.unpack_a(da_o)).max() / np.abs(O.unpack_a(da_o)).max()
    return res


def sphere(n=8, seed=1):
    rng = np.random.default_rng(seed)
    p = W.make_problem(n, n, n, 5e-9, W.sphere_mask(n, n, n), Ms=1.4e5, B0=(0.01, 0, 0.18),
                       omega=[TP * 5e9], kappa=[TP * 2e6], g_re=[TP * 50e6], g_im=[0.0],
                       m0=W.random_state(1, n, n, n, seed, spread=0.3),
                       a0=np.array([2e-3 + 1e-3j]))
    return p.replace(full_demag=True, dt_max=W.stable_dt_max(p))


def holed_box():
    nx, ny, nz = 13, 10, 6
    p = W.make_problem(nx, ny, nz, 4e-9, W.random_mask(nx, ny, nz, 0.75, 5), Ms=1.4e5,
                       Ku=-500.0, ku_axis=(0.0, 0.6, 0.8), B0=(0.02, 0.0, 0.15),
                       omega=TP * np.array([5e9, 5.1e9]), kappa=TP * np.full(2, 2e6),
                       g_re=TP * np.array([40e6, 20e6]), g_im=TP * np.array([0.0, 5e6]),
                       m0=W.random_state(1, nx, ny, nz, 6, spread=0.4),
                       a0=np.array([1e-3, 2e-3j]))
    return p.replace(full_demag=True, dt_max=W.stable_dt_max(p))


def film():
    nx, ny, nz = 24, 20, 2
    p = W.make_problem(nx, ny, nz, (3e-9, 3e-9, 2e-9), W.full_mask(nx, ny, nz), Ms=1.4e5,
                       B0=(0.0, 0.0, 0.3), m0=W.random_state(1, nx, ny, nz, 8, spread=0.2))
    return p.replace(full_demag=True, dt_max=W.stable_dt_max(p))


def afm():
    nx, ny, nz = 10, 8, 4
    p = W.make_problem(nx, ny, nz, 2e-9, W.sphere_mask(nx, ny, nz, 7.0), nsub=2, Ms=4e5,
                       Aex=5e-12, alpha=2e-3, Ku=5e4, B0=(0, 0, 1.0), BE=50.0,
                       omega=[W.afm_params()["w_minus"]], kappa=[TP * 2e6], g_re=[TP * 30e6],
                       g_im=[TP * 30e6], m0=W.random_state(2, nx, ny, nz, 9, 0.1, afm=True),
                       a0=np.array([1e-3j]))
    return p.replace(full_demag=True, dt_max=W.stable_dt_max(p))


@pytest.mark.parametrize("case", ["sphere8", "sphere16", "holed_box", "film", "afm"])
def test_full_demag_rhs_matches_oracle(case):
    p = {"sphere8": lambda: sphere(8), "sphere16": lambda: sphere(16, 2),
         "holed_box": holed_box, "film": film, "afm": afm}[case]()
    r = rhs_compare(p)
    assert r["err_m"] < 2e-6, r
    if "err_da" in r:
        assert r["err_da"] < 1e-6, r


@pytest.mark.parametrize("case", ["sphere8", "holed_box"])
def test_full_demag_replay_1000_steps(case):
    p = {"sphere8": lambda: sphere(8, 3), "holed_box": holed_box}[case]()
    p = p.replace(m0=W.tilted_state(1, p.nx, p.ny, p.nz, 3.0, 0.4), T=1e-6)
    dm, da, info = replay_compare(p, 1000)
    assert info["tiling"]["blocks"] >= 1 and info["tiling"]["bx"] > 0   # tiled kernel
    assert dm <= TOL_M and da <= TOL_A, (dm, da, info["derr"])


def test_switching_back_to_diagonal_factors():
    p = f32_state(sphere(8, 4).replace(full_demag=False, Ndemag=np.array([0.3, 0.3, 0.4])))
    m = np.asarray(p.m0, np.float32)
    plain = sim_for(p, log_cap=0)
    d0, a0, _ = plain.eval_rhs(m, p.a0)
    plain.close()
    sim = sim_for(p, log_cap=0)
    sim.set_demag(True)
    d1, _, _ = sim.eval_rhs(m, p.a0)
    sim.set_demag(False)
    d2, a2, _ = sim.eval_rhs(m, p.a0)
    sim.close()
    assert np.abs(d1 - d0).max() > 1e-3 * np.abs(d0).max()   # the full field differs
    assert np.array_equal(d2, d0) and np.array_equal(a2, a0)


def test_full_demag_rejections():
    p = sphere(8, 5)
    sim = sim_for(p, log_cap=16)
    with pytest.raises(cmx.CmxError) as ei:
        sim.adjoint_record(4, 100)
    assert ei.value.code == cmx.EINVAL
    sim.close()
    big = W.make_problem(200, 4, 4, 5e-9, W.full_mask(200, 4, 4))
    sim = sim_for(big, log_cap=0)
    with pytest.raises(cmx.CmxError) as ei:
        sim.set_demag(True)
    assert ei.value.code == cmx.EINVAL
    sim.close()
