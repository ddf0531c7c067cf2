"""cmx_eval_rhs_noalloc: the right-hand side without any device allocation (needs a B300).

Callers that cannot allocate device memory (plug-ins inside a host program whose allocator owns
all device memory, services under a fixed device-memory budget) use this entry point; its
scratch is one fixed device array inside the library.  The tests call it through the C ABI
twice in a row on different inputs and compare each result with cmx_eval_rhs, which allocates
its own buffers, and with the FP64 oracle, within the tolerance of the other per-stage tests:
profiles from host memory and from device memory, two sublattices, and a problem that just fits
the fixed scratch.  This file is collected last.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import cmx
from paper_2603_03706_b300 import workloads as W

pytestmark = pytest.mark.gpu
TP = 2 * math.pi


def problem(seed, nsub=1, n=None):
    nx, ny, nz = (29, 17, 9) if n is None else (n, n, n)
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1, 1, (2, nz, ny, nx)).astype(np.float32)
    mask = W.sphere_mask(nx, ny, nz, 15.0) if n is None else W.full_mask(nx, ny, nz)
    kw = dict(omega=TP * np.array([5e9, 5.2e9]), kappa=TP * np.array([2e6, 3e6]),
              g_re=TP * np.array([50e6, 30e6]), g_im=TP * np.array([0.0, 10e6]), u=u)
    if nsub == 2:
        p = W.make_problem(nx, ny, nz, 2e-9, mask, nsub=2, Ms=4e5, Aex=5e-12, alpha=2e-3,
                           Ku=5e4, B0=(0, 0, 1.0), Nd=(0, 0, 1), BE=50.0, **kw)
    else:
        p = W.make_problem(nx, ny, nz, 5e-9, mask, Ku=-600.0, B0=(0.01, 0, 0.18),
                           Nd=(0.3, 0.3, 0.4), **kw)
    m = W.random_state(nsub, nx, ny, nz, seed + 100, spread=0.2, afm=(nsub == 2))
    m = m.astype(np.float32).astype(np.float64)
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    return p.replace(m0=m, a0=np.array([3e-3 - 1e-3j, 2e-3j]))


def check_call(p, u_on_device):
    torch = pytest.importorskip("torch")
    m = torch.from_numpy(np.asarray(p.m0, np.float32).copy()).cuda()
    dm = torch.full_like(m, float("nan"))
    u_dev = torch.from_numpy(np.asarray(p.u, np.float32).copy()).cuda() if u_on_device else None
    da, mm = cmx.eval_rhs_noalloc(p, m, dm, a=p.a0, u_dev=u_dev)
    torch.cuda.synchronize()
    got = dm.cpu().numpy().reshape(p.nsub, 3, -1)
    # the allocating entry point on the same inputs
    sim = cmx.Simulation.from_problem(p)
    dm_ref, da_ref, mm_ref = sim.eval_rhs(np.asarray(p.m0, np.float32), p.a0)
    sim.close()
    dm_ref = dm_ref.reshape(p.nsub, 3, -1)
    scale = np.abs(dm_ref).max()
    assert np.abs(got - dm_ref).max() <= 2e-6 * scale
    assert np.abs(da - da_ref).max() <= 1e-6 * np.abs(da_ref).max()
    assert np.abs(mm - mm_ref).max() <= 1e-7
    # the FP64 oracle on the same (FP32-representable) inputs
    op = O.OracleProblem(p.replace(u=np.asarray(p.u, np.float32)))
    dm_o, da_o, mm_o = O.rhs(op, op.m0(), O.pack_a(p.a0))
    dm_o = dm_o.reshape(p.nsub, 3, -1)
    on = p.mask.reshape(-1) > 0
    assert np.abs(got[:, :, on] - dm_o[:, :, on]).max() <= 2e-6 * np.abs(dm_o[:, :, on]).max()
    assert np.abs(got[:, :, ~on]).max(initial=0.0) == 0.0
    assert np.abs(mm - O.unpack_a(mm_o)).max() <= 1e-7
    da_o = O.unpack_a(da_o)
    assert np.abs(da - da_o).max() <= 1e-6 * np.abs(da_o).max()


@pytest.mark.parametrize("case", ["host_profiles", "device_profiles", "two_sublattices"])
def test_noalloc_matches_allocating_rhs_and_oracle_two_calls_in_a_row(case):
    for seed in (1, 2):
        p = problem(seed, nsub=2 if case == "two_sublattices" else 1)
        check_call(p, u_on_device=(case == "device_profiles"))


def test_noalloc_problem_that_just_fits_the_scratch():
    """A full 72^3 box with two profiled modes (host profiles): compact layout, profiles, state,
    slope and the dense profile copy take about 16.5 MB of the 16 MiB array."""
    check_call(problem(3, n=72), u_on_device=False)


def test_noalloc_rejects_problems_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    for n, prof in ((96, False), (73, True)):
        p = problem(4, n=n) if prof else W.make_problem(
            n, n, n, 5e-9, W.full_mask(n, n, n), omega=[TP * 5e9], kappa=[0.0], g_re=[0.0],
            g_im=[0.0])
        m = torch.zeros((p.nsub, 3, n, n, n), dtype=torch.float32, device="cuda")
        dm = torch.zeros_like(m)
        with pytest.raises(cmx.CmxError) as ei:
            cmx.eval_rhs_noalloc(p, m, dm, a=p.a0)
        assert ei.value.code == cmx.ESCRATCH
