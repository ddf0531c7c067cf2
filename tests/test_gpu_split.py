"""Operator-split scheme on the GPU (needs a B300): against the FP64 oracle's split scheme, and
its first-order convergence to the coupled solution (the paper's Sec. V scaling)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

from gpu_util import f32_state, masked

pytestmark = pytest.mark.gpu


def sphere():
    return f32_state(W.single_sphere().replace(dt_max=2e-13))


def run_gpu(p, T, ds=None):
    sim = cmx.Simulation.from_problem(p, log_cap=0)
    if ds:
        sim.set_split(ds)
    sim.run(T)
    out = sim.get_a(), sim.get_m(), sim.sync()
    sim.close()
    return out


def test_split_matches_the_oracle_split():
    p = sphere()
    T, ds = 1.0e-9, 2e-12
    a, m, st = run_gpu(p, T, ds)
    assert abs(st["t"] - T) < 1e-21
    it = O.Integrator(O.OracleProblem(p))
    rc, _ = it.run_split(T, ds)
    assert rc == 0
    o = it.state()
    m_o = o["m"].reshape(1, 3, p.nz, p.ny, p.nx)
    assert np.abs(a - o["a"]).max() <= 2e-3 * np.abs(o["a"]).max(), (a, o["a"])
    assert np.abs(masked(p, m) - masked(p, m_o)).max() <= 1e-4


def test_split_converges_at_first_order():
    p = sphere()
    T = 1.0e-9
    a_ref, _, _ = run_gpu(p, T)
    errs = []
    for ds in (4e-12, 2e-12, 1e-12):
        a, _, _ = run_gpu(p, T, ds)
        errs.append(np.abs(a - a_ref).max() / np.abs(a_ref).max())
    assert 1.6 < errs[0] / errs[1] < 2.5 and 1.6 < errs[1] / errs[2] < 2.5, errs


def test_split_off_again_and_adjoint_refuses_it():
    p = sphere()
    sim = cmx.Simulation.from_problem(p, log_cap=64)
    sim.set_split(2e-12)
    with pytest.raises(cmx.CmxError):
        sim.adjoint_record(10, 100)
    sim.run(0.1e-9)
    sim.set_split(0.0)
    st = sim.run(0.2e-9)
    assert abs(st["t"] - 0.2e-9) < 1e-21
    sim.close()
