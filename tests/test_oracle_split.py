"""Pins of the oracle's operator-split scheme (the paper's Python tier, Sec. III B/C), CPU only.

* Against the coupled Dormand-Prince solution its global error falls linearly with the split
  interval (first order: the commutator of the cavity and magnet steps, Sec. V).
* Decoupled (g = 0) the cavity step is a classical RK4 step: a driven free cavity converges at
  fourth order to its closed form, and the magnet follows the coupled solution exactly.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2603_03706_b300 import workloads as W

from test_oracle_drive import closed_form, free_cavity

TP = 2 * math.pi


def resonant_sphere():
    p = W.single_sphere().replace(rtol=1e-10, dt_max=2e-13)
    return p


def test_split_error_is_first_order_in_the_interval():
    p = resonant_sphere()
    T = 1.0e-9
    ref = O.Integrator(O.OracleProblem(p))
    rc, _ = ref.run(T)
    assert rc == 0
    a_ref = ref.state()["a"]
    errs = []
    for ds in (4e-12, 2e-12, 1e-12):
        it = O.Integrator(O.OracleProblem(p))
        rc, _ = it.run_split(T, ds)
        assert rc == 0
        st = it.state()
        assert abs(st["t"] - T) < 1e-21
        errs.append(np.abs(st["a"] - a_ref).max() / np.abs(a_ref).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 < r1 < 2.5 and 1.6 < r2 < 2.5, errs
    assert errs[0] < 0.2


def test_decoupled_split_is_rk4_for_the_cavity():
    p = free_cavity(drive=[3e7 + 1e7j, -2e7j], a0=(1e-3 + 2e-4j, 0), rtol=1e-10)
    T = 0.3e-9
    errs = []
    for ds in (4e-12, 2e-12):
        it = O.Integrator(O.OracleProblem(p))
        rc, _ = it.run_split(T, ds)
        assert rc == 0
        errs.append(np.abs(it.state()["a"] - closed_form(p, T)).max())
    assert 12.0 < errs[0] / errs[1] < 20.0, errs   # 2^4 = 16


def test_decoupled_split_leaves_the_magnet_unchanged():
    p = resonant_sphere().replace(g_re=np.array([0.0]), g_im=np.array([0.0]))
    T = 0.5e-9
    a = O.Integrator(O.OracleProblem(p))
    a.run(T)
    b = O.Integrator(O.OracleProblem(p))
    rc, _ = b.run_split(T, 3e-12)
    assert rc == 0
    assert np.abs(a.state()["m"] - b.state()["m"]).max() < 1e-8
