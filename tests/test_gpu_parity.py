"""Parity of the CUDA integrator with the FP64 oracle (needs a B300).

* single right-hand-side evaluations (one stage) on grids whose tiles are partly empty, with a
  ragged tail in every direction, holes in the mask, two sublattices and up to 8 modes;
* 1000 adaptive GPU steps replayed step for step by the oracle: max|dm| <= 2e-5 and
  |da|/max|a| <= 1e-4;
* the full-size workloads in their measured launch configuration on sampled outputs;
* edge cases (one cell, no modes, every tile an edge tile), determinism, error statuses.
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


def ragged_problem(nsub=1, nmodes=2, holes=False, seed=0):
    nx, ny, nz = 37, 21, 11
    mask = W.random_mask(nx, ny, nz, 0.8, seed) if holes else W.sphere_mask(nx, ny, nz, 19.0)
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (nmodes, nz, ny, nx)).astype(np.float32) if nmodes else None
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
    # non-uniform drive and state: keep every exchange mode inside the stability region
    return p.replace(dt_max=W.stable_dt_max(p))


def rhs_compare(p, tiling=None):
    p = f32_state(f32_profiles(p))
    sim = sim_for(p, log_cap=0, tiling=tiling)
    dm_g, da_g, mm_g = sim.eval_rhs(np.asarray(p.m0, np.float32), p.a0)
    sim.close()
    op = O.OracleProblem(p)
    dm_o, da_o, mm_o = O.rhs(op, op.m0(), O.pack_a(p.a0))
    dm_o = dm_o.reshape(p.nsub, 3, p.nz, p.ny, p.nx)
    scale = np.abs(masked(p, dm_o)).max()
    err_m = np.abs(masked(p, dm_g) - masked(p, dm_o)).max() / scale
    outside = np.abs(dm_g.reshape(p.nsub, 3, -1)[:, :, p.mask.reshape(-1) == 0]).max(initial=0.0)
    res = dict(err_m=err_m, outside=outside)
    if p.nmodes:
        mm_o = O.unpack_a(mm_o)
        da_o = O.unpack_a(da_o)
        res["err_mm"] = np.abs(mm_g - mm_o).max()
        res["err_da"] = np.abs(da_g - da_o).max() / np.abs(da_o).max()
    return res


# ---------------------------------------------------------------------------------------------
# one stage
# ---------------------------------------------------------------------------------------------

# tiles (bx, by, bz[, blocks_per_sm]): shapes, fewest planes per block (segments cut across
# columns), one resident block per SM (many segments per block)
TILINGS = [None, (32, 8, 3), (32, 4, 5), (32, 16, 11), (32, 8, 1), (32, 4, 1), (32, 16, 1),
           (32, 8, 2, 1), (32, 4, 7, 1)]


@pytest.mark.parametrize("tiling", TILINGS)
def test_rhs_ferromagnet_ragged(tiling):
    r = rhs_compare(ragged_problem(), tiling)
    assert r["err_m"] < 2e-6, r
    assert r["outside"] == 0.0
    assert r["err_mm"] < 1e-7 and r["err_da"] < 1e-6, r


@pytest.mark.parametrize("tiling", [(32, 4, 4), (32, 16, 2)])
def test_rhs_mask_with_holes_and_many_runs_per_row(tiling):
    r = rhs_compare(ragged_problem(holes=True, nmodes=8, seed=3), tiling)
    assert r["err_m"] < 2e-6 and r["outside"] == 0.0, r
    assert r["err_mm"] < 1e-7 and r["err_da"] < 1e-6, r


@pytest.mark.parametrize("tiling", [(32, 8, 4), (32, 4, 2)])
def test_rhs_antiferromagnet_two_sublattices(tiling):
    r = rhs_compare(ragged_problem(nsub=2, nmodes=2, seed=5), tiling)
    assert r["err_m"] < 2e-6, r
    assert r["err_mm"] < 1e-7 and r["err_da"] < 1e-6, r


def test_rhs_no_modes_single_cell():
    p = W.make_problem(1, 1, 1, 5e-9, W.full_mask(1, 1, 1), B0=(0.02, 0, 0.2),
                       m0=W.tilted_state(1, 1, 1, 1, 30.0, 0.4))
    r = rhs_compare(p)
    assert r["err_m"] < 1e-6


# ---------------------------------------------------------------------------------------------
# 1000 replayed steps
# ---------------------------------------------------------------------------------------------

def test_replay_single_sphere_1000_steps():
    dm, da, info = replay_compare(W.single_sphere(), 1000)
    assert info["stats"]["accepted"] >= 990
    assert dm <= TOL_M and da <= TOL_A, (dm, da)


@pytest.mark.parametrize("tiling", [(32, 4, 4), (32, 16, 2)])
def test_replay_ragged_multimode_1000_steps(tiling):
    p = ragged_problem(nmodes=3, seed=11)
    p = p.replace(m0=W.tilted_state(1, p.nx, p.ny, p.nz, 5.0, 0.3), a0=np.array([1e-3, 0, 0j]))
    dm, da, info = replay_compare(p.replace(T=1e-6), 1000, tiling=tiling)
    assert dm <= TOL_M and da <= TOL_A, (dm, da)


def test_replay_afm_complex_coupling_1000_steps():
    p = ragged_problem(nsub=2, nmodes=2, seed=13)
    m = W.tilted_state(2, p.nx, p.ny, p.nz, 1.0, 0.0, afm=True)
    p = p.replace(m0=m, a0=np.zeros(2, complex), u=None, T=1e-6)
    for tiling in ((32, 8, 4), (32, 4, 1)):
        dm, da, info = replay_compare(p, 1000, tiling=tiling)
        assert dm <= TOL_M and da <= TOL_A, (tiling, dm, da)


# ---------------------------------------------------------------------------------------------
# single-block integrator (small grids: the whole state in one block's shared memory)
# ---------------------------------------------------------------------------------------------

def small_afm():
    nx, ny, nz = 10, 9, 4
    p = W.make_problem(nx, ny, nz, 2e-9, W.full_mask(nx, ny, nz), nsub=2, Ms=4e5, Aex=5e-12,
                       alpha=2e-3, Ku=5e4, B0=(0, 0, 1.0), Nd=(0, 0, 1), BE=50.0,
                       omega=[W.afm_params()["w_minus"] - TP * 60e6] * 2,
                       kappa=[TP * 2e6] * 2, g_re=[TP * 30e6] * 2, g_im=[0.0, TP * 30e6],
                       m0=W.random_state(2, nx, ny, nz, 31, spread=0.05, afm=True), T=1e-6)
    return p.replace(dt_max=W.stable_dt_max(p))


def small_profiled():
    nx, ny, nz = 11, 9, 7
    rng = np.random.default_rng(41)
    u = rng.uniform(-1, 1, (3, nz, ny, nx)).astype(np.float32)
    p = W.make_problem(nx, ny, nz, 5e-9, W.random_mask(nx, ny, nz, 0.8, 41), Ku=-610.0,
                       ku_axis=(0.6, 0.0, 0.8), B0=(0.01, 0, 0.187), Nd=(0.3, 0.3, 0.4),
                       omega=TP * np.array([4.9e9, 5.0e9, 5.1e9]), kappa=TP * np.full(3, 2e6),
                       g_re=TP * np.array([40e6, 60e6, 20e6]), g_im=TP * np.array([0, 10e6, 0]),
                       u=u, m0=W.tilted_state(1, nx, ny, nz, 5.0, 0.3),
                       a0=np.array([1e-3, 0, 2e-4j]), T=1e-6)
    return p.replace(dt_max=W.stable_dt_max(p))


@pytest.mark.parametrize("case", ["sphere", "afm", "profiles_holes"])
def test_single_block_integrator_1000_steps(case):
    """Grids that fit one block's shared memory run on the single-block integrator by default:
    1000 adaptive attempts replayed by the oracle (error norms and step sizes checked)."""
    p = {"sphere": W.single_sphere, "afm": small_afm, "profiles_holes": small_profiled}[case]()
    dm, da, info = replay_compare(p, 1000)
    assert info["tiling"]["blocks"] == 1 and info["tiling"]["bx"] == 0, info["tiling"]
    assert dm <= TOL_M and da <= TOL_A, (dm, da, info["derr"])


def boundary_problem(ncells, nsub):
    """A 10 x 8 x 4 box whose first `ncells` cells (x fastest) are magnetic: 288 cells is the
    largest grid whose cells the single-block integrator keeps one per worker thread in
    registers, 289 the smallest that takes the shared-memory form."""
    nx, ny, nz = 10, 8, 4
    mask = np.zeros(nx * ny * nz, np.uint8)
    mask[:ncells] = 1
    mask = mask.reshape(nz, ny, nx)
    rng = np.random.default_rng(ncells + 7 * nsub)
    u = rng.uniform(-1, 1, (2, nz, ny, nx)).astype(np.float32)
    kw = dict(omega=TP * np.array([4.95e9, 5.05e9]), kappa=TP * np.array([2e6, 3e6]),
              g_re=TP * np.array([40e6, 30e6]), g_im=TP * np.array([0.0, 15e6]), u=u,
              a0=np.array([1e-3, 5e-4j]), T=1e-6)
    if nsub == 2:
        p = W.make_problem(nx, ny, nz, 2e-9, mask, nsub=2, Ms=4e5, Aex=5e-12, alpha=2e-3,
                           Ku=5e4, B0=(0, 0, 1.0), Nd=(0, 0, 1), BE=50.0,
                           m0=W.random_state(2, nx, ny, nz, 3, spread=0.05, afm=True), **kw)
    else:
        p = W.make_problem(nx, ny, nz, 5e-9, mask, Ku=-610.0, ku_axis=(0.6, 0.0, 0.8),
                           B0=(0.01, 0, 0.187), Nd=(0.3, 0.3, 0.4),
                           m0=W.tilted_state(1, nx, ny, nz, 4.0, 0.2), **kw)
    return p.replace(dt_max=W.stable_dt_max(p))


@pytest.mark.parametrize("nsub", [1, 2])
@pytest.mark.parametrize("ncells", [288, 289])
def test_single_block_register_and_shared_forms(ncells, nsub):
    """Both forms of the single-block integrator at the boundary between them (288 cells: one
    cell per worker, state in registers; 289: cells in shared memory), with profiles and a
    complex coupling: 1000 replayed attempts against the oracle."""
    p = boundary_problem(ncells, nsub)
    assert int(p.mask.sum()) == ncells
    dm, da, info = replay_compare(p, 1000)
    assert info["tiling"]["blocks"] == 1 and info["tiling"]["bx"] == 0, info["tiling"]
    assert dm <= TOL_M and da <= TOL_A, (dm, da, info["derr"])


def test_single_block_and_tiled_kernels_agree():
    """The same 8^3 sphere on the single-block integrator and on the tiled multi-block kernel
    (tile forced): both replays match the oracle."""
    p = W.single_sphere()
    dm1, da1, i1 = replay_compare(p, 400)
    dm2, da2, i2 = replay_compare(p, 400, tiling=(32, 4, 2))
    assert i1["tiling"]["blocks"] == 1 and i2["tiling"]["blocks"] > 1
    for dm, da in ((dm1, da1), (dm2, da2)):
        assert dm <= TOL_M and da <= TOL_A, (dm, da)


def test_single_block_split_scheme_matches_tiled():
    """Operator-split mode on the single-block integrator against the tiled kernel."""
    p = f32_state(W.single_sphere(T=0.2e-9).replace(a0=np.array([1e-2 + 0j])))
    out = []
    for tiling in (None, (32, 4, 2)):
        sim = sim_for(p, log_cap=0, tiling=tiling)
        sim.set_split(2e-12)
        sim.run(p.T)
        out.append((sim.get_m(), sim.get_a(), sim.get_tiling()["blocks"]))
        sim.close()
    assert out[0][2] == 1 and out[1][2] > 1
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-5
    assert np.abs(out[0][1] - out[1][1]).max() < 1e-5 * np.abs(out[1][1]).max()


# ---------------------------------------------------------------------------------------------
# full-size workloads in the measured configuration (sampled)
# ---------------------------------------------------------------------------------------------

def test_full_size_multimode_sphere_rhs():
    p = W.multimode_sphere()
    r = rhs_compare(p)
    assert r["err_m"] < 2e-6 and r["err_mm"] < 1e-7 and r["err_da"] < 1e-6, r


def test_full_size_multimode_sphere_1000_steps():
    """The 128x128x64 sphere (137,376 cells, four profiled modes) in the benchmark's launch
    configuration (window picked by the autotuner, every resident block, several segments per
    block): 1000 adaptive device attempts replayed by the oracle, with the error norms and the
    step-size sequence checked attempt by attempt."""
    dm, da, info = replay_compare(W.multimode_sphere(), 1000, autotune=5)
    assert info["stats"]["accepted"] >= 900
    assert info["tiling"]["blocks"] > 100, info["tiling"]
    assert dm <= TOL_M and da <= TOL_A, (dm, da, info["derr"], info["tiling"])


def test_full_size_afm_film_rhs():
    p = W.afm_film()
    r = rhs_compare(p.replace(m0=W.random_state(2, p.nx, p.ny, p.nz, 7, 0.1, afm=True)))
    assert r["err_m"] < 2e-6 and r["err_mm"] < 1e-7 and r["err_da"] < 1e-6, r


def test_full_size_afm_film_200_steps():
    """The 256x256x16 two-sublattice film (complex coupling of mode 2) in the benchmark's launch
    configuration: 200 adaptive device attempts replayed by the oracle."""
    dm, da, info = replay_compare(W.afm_film(), 200, autotune=3)
    assert info["stats"]["accepted"] >= 150
    assert dm <= TOL_M and da <= TOL_A, (dm, da, info["derr"], info["tiling"])


# ---------------------------------------------------------------------------------------------
# properties
# ---------------------------------------------------------------------------------------------

def test_deterministic_bitwise():
    p = f32_state(ragged_problem(seed=21).replace(T=1e-6))
    outs = []
    for _ in range(2):
        sim = sim_for(p, log_cap=64)
        sim.run(p.T, max_attempts=50)
        outs.append((sim.get_m(), sim.get_a(), sim.get_log()["dt"]))
        sim.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


def test_run_lands_on_T_and_resumes():
    p = W.single_sphere(T=0.2e-9)
    sim = sim_for(p, log_cap=0)
    sim.set_launch_attempts(7)                  # many short launches
    st = sim.run(0.1e-9)
    assert st["t"] == pytest.approx(0.1e-9, abs=0) or abs(st["t"] - 0.1e-9) < 1e-24
    st = sim.run(0.2e-9)
    assert abs(st["t"] - 0.2e-9) < 1e-24
    assert st["launches"] > 2
    sim.close()


def test_unit_norm_after_steps():
    p = ragged_problem(seed=4).replace(T=1e-6)
    sim = sim_for(p, log_cap=0)
    sim.run(p.T, max_attempts=200)
    m = masked(p, sim.get_m())
    n = np.linalg.norm(m, axis=1)
    assert np.abs(n - 1).max() < 1e-6
    sim.close()


def test_barrier_timeout_status_and_recovery():
    """A block that leaves without arriving makes the others hit their wait limit: the run
    returns CMX_ETIMEOUT, the context stays usable, set_state clears the error."""
    p = ragged_problem(seed=8).replace(T=1e-6)
    sim = sim_for(p, log_cap=0)
    sim.set_timeout(1_000_000)                  # 1 ms
    sim.debug_skip_arrival(0)
    with pytest.raises(cmx.CmxError) as ei:
        sim.run(p.T, max_attempts=10)
    assert ei.value.code == cmx.ETIMEOUT
    assert sim.status() == cmx.ETIMEOUT        # sticky
    sim.set_state(p.m0, p.a0)
    st = sim.run(p.T, max_attempts=10)
    assert st["attempts"] == 10 and st["status"] == 0
    sim.close()


def test_nan_state_reports_enan():
    p = ragged_problem(seed=9).replace(T=1e-6)
    m = np.array(p.m0)
    m[0, 0, 5, 10, 18] = np.nan
    sim = sim_for(p, log_cap=0)
    sim.set_state(m, p.a0)
    with pytest.raises(cmx.CmxError) as ei:
        sim.run(p.T, max_attempts=5)
    assert ei.value.code == cmx.ENAN
    sim.close()


def test_autotune_restores_the_state_and_keeps_a_compiled_window():
    p = f32_state(f32_profiles(ragged_problem(nmodes=2, seed=21)))
    sim = sim_for(p, log_cap=64)
    sim.run(p.T, max_attempts=5)
    m0, a0, st0 = sim.get_m(), sim.get_a(), sim.sync()
    t = sim.autotune(3)
    assert (t["bx"], t["by"]) in ((32, 4), (32, 8), (32, 16))
    us = t["us_per_attempt"]
    assert all(us[k] > 0 for k in ("32x4", "32x8", "32x16")), t
    assert us["single_block"] != us["single_block"], t   # NaN: the grid is too large for it
    st1 = sim.sync()
    assert np.array_equal(sim.get_m(), m0) and np.array_equal(sim.get_a(), a0)
    assert (st1["t"], st1["attempts"], st1["accepted"]) == (st0["t"], st0["attempts"],
                                                            st0["accepted"])
    sim.run(p.T, max_attempts=5)
    assert sim.sync()["attempts"] == st0["attempts"] + 5
    sim.close()


@pytest.mark.parametrize("case", ["ragged", "single_block", "afm", "dense_afm"])
def test_save_and_load_state_resume_bitwise(case):
    """A run saved after some attempts and resumed in a fresh handle continues bitwise like the
    uninterrupted run: state, cavity amplitudes, step sizes and the step log (the dense case runs
    on the tensor-copy path of grids magnetic over their whole box)."""
    if case == "ragged":
        p = f32_state(ragged_problem(seed=17).replace(T=1e-6))
    elif case == "afm":
        p = f32_state(ragged_problem(nsub=2, seed=19).replace(T=1e-6))
    elif case == "dense_afm":
        p = ragged_problem(nsub=2, seed=29)
        p = p.replace(mask=W.full_mask(p.nx, p.ny, p.nz), T=1e-6)
        p = f32_state(p.replace(dt_max=W.stable_dt_max(p)))
    else:
        p = f32_state(W.single_sphere())
    sim = sim_for(p, log_cap=400)
    sim.run(p.T, max_attempts=120)
    blob = sim.save_state()
    sim.run(p.T, max_attempts=150)
    ref = (sim.get_m(), sim.get_a(), sim.sync(), sim.get_log())
    sim.close()
    sim = sim_for(p, log_cap=400)
    sim.load_state(blob)
    sim.run(p.T, max_attempts=150)
    got = (sim.get_m(), sim.get_a(), sim.sync(), sim.get_log())
    sim.close()
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    assert (ref[2]["t"], ref[2]["attempts"], ref[2]["accepted"]) == \
        (got[2]["t"], got[2]["attempts"], got[2]["accepted"])
    n = ref[3]["n"]
    assert got[3]["n"] == n
    assert np.array_equal(ref[3]["dt"][120:n], got[3]["dt"][120:n])


def test_load_state_rejects_another_problem():
    p = ragged_problem(seed=23)
    sim = sim_for(p, log_cap=0)
    blob = sim.save_state()
    sim.close()
    q = W.single_sphere()
    other = sim_for(q, log_cap=0)
    with pytest.raises(cmx.CmxError) as ei:
        other.load_state(blob)
    assert ei.value.code == cmx.EINVAL
    with pytest.raises(cmx.CmxError):
        other.load_state(blob[:10])
    other.close()
