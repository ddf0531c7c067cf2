"""cmx_eval_rhs_noalloc: the right-hand side without any device allocation (needs a B300).

Callers that cannot allocate device memory (code running during stream capture, plug-ins in a
host program that owns the allocator, fixed memory budgets) use this entry point; its scratch
is one fixed device array inside the library.  The test calls it through the C ABI twice in a
row on different inputs and compares each result with cmx_eval_rhs, which allocates its own
buffers, within the tolerance of the other per-stage tests.  This file is collected last.
"""
import math

import numpy as np
import pytest

from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


def problem(seed):
    nx, ny, nz = 29, 17, 9
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (2, nz, ny, nx)).astype(np.float32)
    p = W.make_problem(nx, ny, nz, 5e-9, W.sphere_mask(nx, ny, nz, 15.0), Ku=-600.0,
                       B0=(0.01, 0, 0.18), Nd=(0.3, 0.3, 0.4), omega=TP * np.array([5e9, 5.2e9]),
                       kappa=TP * np.array([2e6, 3e6]), g_re=TP * np.array([50e6, 30e6]),
                       g_im=TP * np.array([0.0, 10e6]), u=u)
    m = W.random_state(1, nx, ny, nz, seed + 100, spread=0.2).astype(np.float32)
    return p.replace(m0=m, a0=np.array([3e-3 - 1e-3j, 2e-3j]))


def test_noalloc_matches_allocating_rhs_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    for seed in (1, 2):
        p = problem(seed)
        m = torch.from_numpy(np.asarray(p.m0, np.float32).copy()).cuda()
        dm = torch.full_like(m, float("nan"))
        da, mm = cmx.eval_rhs_noalloc(p, m, dm, a=p.a0)
        torch.cuda.synchronize()
        sim = cmx.Simulation.from_problem(p)
        dm_ref, da_ref, mm_ref = sim.eval_rhs(np.asarray(p.m0, np.float32), p.a0)
        sim.close()
        got = dm.cpu().numpy()
        scale = np.abs(dm_ref).max()
        assert np.abs(got - dm_ref).max() <= 2e-6 * scale
        assert np.abs(da - da_ref).max() <= 1e-6 * np.abs(da_ref).max()
        assert np.abs(mm - mm_ref).max() <= 1e-7


def test_noalloc_rejects_problems_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    n = 96
    p = W.make_problem(n, n, n, 5e-9, W.full_mask(n, n, n), omega=[TP * 5e9], kappa=[0.0],
                       g_re=[0.0], g_im=[0.0])
    m = torch.zeros((1, 3, n, n, n), dtype=torch.float32, device="cuda")
    dm = torch.zeros_like(m)
    with pytest.raises(cmx.CmxError) as ei:
        cmx.eval_rhs_noalloc(p, m, dm)
    assert ei.value.code == cmx.ESCRATCH
