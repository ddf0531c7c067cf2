"""Pins of the oracle's full magnetostatic demag (CPU only).

The cell-pair tensor of Newell, Williams & Dunlop (1993) and the direct-sum field are checked
against what the mathematics fixes without them:
* a cube's self term is 1/3 on the diagonal and 0 off it; any cell's self term has trace 1;
* away from the source cell the tensor is traceless (Laplace) and has the parity of a dipole
  field (xx, yy, zz even; xy odd in x and y);
* far from the source it tends to the point-dipole tensor (delta R^2 - 3 r r) / (4 pi R^5) V;
* summed over all cell pairs of a cuboid of cells it gives the demag factors of the cuboid,
  Aharoni's closed form (J. Appl. Phys. 83, 3432 (1998)), which itself is pinned by the cube's
  1/3 and by D_x + D_y + D_z = 1;
* the field of a uniformly magnetised cuboid averaged over its cells is -mu0 Ms D m with those
  factors, and the right-hand side with full demag reduces to the diagonal-factor one for that
  averaged field on a single cell.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2603_03706_b300 import workloads as W


def aharoni_dz(a, b, c):
    """Demag factor along z of a 2a x 2b x 2c rectangular prism (Aharoni 1998, Eq. (1))."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    t = (b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
    t += (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
    t += b / (2 * c) * math.log((ab + a) / (ab - a))
    t += a / (2 * c) * math.log((ab + b) / (ab - b))
    t += c / (2 * a) * math.log((bc - b) / (bc + b))
    t += c / (2 * b) * math.log((ac - a) / (ac + a))
    t += 2 * math.atan(a * b / (c * r))
    t += (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
    t += (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
    t += c / (a * b) * (ac + bc)
    t -= (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c)
    return t / math.pi


def aharoni(a, b, c):
    return np.array([aharoni_dz(b, c, a), aharoni_dz(c, a, b), aharoni_dz(a, b, c)])


def test_aharoni_closed_form_is_consistent():
    assert aharoni(1, 1, 1) == pytest.approx([1 / 3] * 3, abs=1e-14)
    for abc in ((1.0, 2.0, 0.5), (3.0, 1.0, 0.2), (0.3, 0.4, 5.0)):
        assert aharoni(*abc).sum() == pytest.approx(1.0, abs=1e-13)
    # thin plate: D_z -> 1; long bar along z: D_z -> 0
    assert aharoni(100, 100, 0.01)[2] > 0.999
    assert aharoni(0.01, 0.01, 100)[2] < 1e-3


def tensor_at(T, nx, ny, nz, i, j, k):
    return T[:, k + nz - 1, j + ny - 1, i + nx - 1]


def test_self_terms():
    T = O.demag_tensor(1, 1, 1, 2e-9, 2e-9, 2e-9)
    assert T[:, 0, 0, 0] == pytest.approx([1 / 3, 1 / 3, 1 / 3, 0, 0, 0], abs=1e-14)
    for c in ((1e-9, 2e-9, 3e-9), (5e-9, 5e-9, 1e-9), (1e-9, 4e-9, 4e-9)):
        s = O.demag_tensor(1, 1, 1, *c)[:, 0, 0, 0]
        assert s[:3].sum() == pytest.approx(1.0, abs=1e-13)
        assert np.abs(s[3:]).max() < 1e-14
        # the shortest side has the largest factor
        assert np.argmax(s[:3]) == int(np.argmin(c))


def test_traceless_and_parity_away_from_the_source():
    nx, ny, nz = 4, 3, 3
    T = O.demag_tensor(nx, ny, nz, 1e-9, 1.5e-9, 2e-9)
    tr = T[0] + T[1] + T[2]
    tr[nz - 1, ny - 1, nx - 1] -= 1.0
    assert np.abs(tr).max() < 1e-12
    # xx, yy, zz even in every displacement; xy odd in x and y, even in z; xz odd in x and z
    for c in range(3):
        assert np.allclose(T[c], T[c][::-1, ::-1, ::-1], atol=1e-15)
    assert np.allclose(T[3], -T[3][:, :, ::-1], atol=1e-15)
    assert np.allclose(T[3], -T[3][:, ::-1, :], atol=1e-15)
    assert np.allclose(T[3], T[3][::-1, :, :], atol=1e-15)
    assert np.allclose(T[4], -T[4][:, :, ::-1], atol=1e-15)
    assert np.allclose(T[4], -T[4][::-1, :, :], atol=1e-15)
    assert np.allclose(T[5], -T[5][:, ::-1, :], atol=1e-15)
    assert np.allclose(T[5], -T[5][::-1, :, :], atol=1e-15)


def test_swapping_axes_swaps_components():
    T = O.demag_tensor(3, 3, 2, 1e-9, 1e-9, 3e-9)
    # square cells in the xy plane: N_yy(X, Y, Z) = N_xx(Y, X, Z), N_yz(X, Y, Z) = N_xz(Y, X, Z)
    assert np.allclose(T[1], np.transpose(T[0], (0, 2, 1)), atol=1e-15)
    assert np.allclose(T[5], np.transpose(T[4], (0, 2, 1)), atol=1e-15)


def test_far_field_is_the_point_dipole():
    n = 13
    c = np.array([1e-9, 1.2e-9, 0.9e-9])
    T = O.demag_tensor(n, n, n, *c)
    V = c.prod()
    for (i, j, k) in ((12, 0, 0), (0, 12, 0), (9, 7, 5), (12, 12, 12), (10, -6, 3)):
        r = np.array([i, j, k]) * c
        R = np.linalg.norm(r)
        dip = (np.eye(3) * R * R - 3 * np.outer(r, r)) / (4 * math.pi * R ** 5) * V
        got = tensor_at(T, n, n, n, i, j, k)
        want = np.array([dip[0, 0], dip[1, 1], dip[2, 2], dip[0, 1], dip[0, 2], dip[1, 2]])
        # the next multipole correction is relative (cell / R)^2
        assert np.abs(got - want).max() <= 0.05 * np.abs(want).max(), (i, j, k)


@pytest.mark.parametrize("shape,cell", [((4, 6, 2), (0.5e-9, 2e-9 / 3, 0.5e-9)),
                                        ((5, 5, 5), (1e-9, 1e-9, 1e-9)),
                                        ((8, 8, 1), (2e-9, 2e-9, 1e-9)),
                                        ((3, 2, 7), (1e-9, 2e-9, 0.5e-9))])
def test_pair_sum_of_a_cuboid_is_aharonis_factor(shape, cell):
    nx, ny, nz = shape
    T = O.demag_tensor(nx, ny, nz, *cell)
    mult = np.einsum("k,j,i->kji", nz - np.abs(np.arange(-(nz - 1), nz)),
                     ny - np.abs(np.arange(-(ny - 1), ny)), nx - np.abs(np.arange(-(nx - 1), nx)))
    avg = (T * mult[None]).reshape(6, -1).sum(axis=1) / (nx * ny * nz)
    half = 0.5 * np.array([nx * cell[0], ny * cell[1], nz * cell[2]])
    assert avg[:3] == pytest.approx(aharoni(*half), abs=1e-12)
    assert np.abs(avg[3:]).max() < 1e-13


def test_uniform_cuboid_field_and_rhs():
    nx, ny, nz = 6, 4, 3
    c = 2e-9
    p = W.make_problem(nx, ny, nz, c, W.full_mask(nx, ny, nz), Ms=1.4e5, B0=(0, 0, 0.2))
    p = p.replace(full_demag=True)
    mdir = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    m = np.broadcast_to(mdir[None, :, None, None, None], (1, 3, nz, ny, nx)).copy()
    op = O.OracleProblem(p.replace(m0=m))
    bd = O.demag_field(op, op.m0())
    D = aharoni(nx * c / 2, ny * c / 2, nz * c / 2)
    want = -W.MU0 * p.Ms * D * mdir
    assert bd.mean(axis=1) == pytest.approx(want, rel=1e-10, abs=1e-14)
    # a single cell: full demag is the diagonal self term
    q = W.make_problem(1, 1, 1, (1e-9, 2e-9, 3e-9), W.full_mask(1, 1, 1), B0=(0.01, 0, 0.2))
    Nself = O.demag_tensor(1, 1, 1, 1e-9, 2e-9, 3e-9)[:3, 0, 0, 0]
    m1 = np.array([0.6, 0.0, 0.8]).reshape(1, 3, 1, 1, 1)
    o_full = O.OracleProblem(q.replace(full_demag=True, m0=m1))
    o_diag = O.OracleProblem(q.replace(Ndemag=Nself, m0=m1))
    d_full, _, _ = O.rhs(o_full, o_full.m0(), np.zeros(0))
    d_diag, _, _ = O.rhs(o_diag, o_diag.m0(), np.zeros(0))
    assert np.allclose(d_full, d_diag, rtol=1e-12, atol=0)
