"""The C-ABI library builds for sm_103a, loads, and exports every function declared in
include/cmx.h (no GPU needed: nothing here calls into the device code)."""
import ctypes
import os
import re

import pytest

from paper_2603_03706_b300 import build, cmx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(cmx_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(cmx.SIGNATURES)
    cmx.load()


def test_status_strings_without_device():
    lib = cmx.load()
    assert lib.cmx_status_string(cmx.ETIMEOUT).decode() == "device wait timed out"
    assert lib.cmx_status_string(cmx.OK).decode() == "ok"


def test_create_rejects_bad_arguments_before_touching_the_device():
    lib = cmx.load()
    h = ctypes.c_void_p()
    g = cmx.Grid(0, 4, 4, 1e-9, 1e-9, 1e-9, 1)          # nx = 0
    m = cmx.Material(1.4e5, 3.7e-12, 1e-3, 1.76e11, 0.0)
    sv = cmx.Solver(1e-6, 1e-3, 1e-13, 1e-18, 1e-11, 0.0, 0, 0)
    mask = (ctypes.c_uint8 * 16)(*([1] * 16))
    assert lib.cmx_create(ctypes.byref(g), mask, ctypes.byref(m), None, ctypes.byref(sv), None,
                          None, ctypes.byref(h)) == cmx.EINVAL
    g = cmx.Grid(4, 4, 1, 1e-9, 1e-9, 1e-9, 3)          # nsub = 3
    assert lib.cmx_create(ctypes.byref(g), mask, ctypes.byref(m), None, ctypes.byref(sv), None,
                          None, ctypes.byref(h)) == cmx.EINVAL
    md = cmx.Modes()
    md.n_modes = 9                                       # more than CMX_MAX_MODES
    g = cmx.Grid(4, 4, 1, 1e-9, 1e-9, 1e-9, 1)
    assert lib.cmx_create(ctypes.byref(g), mask, ctypes.byref(m), ctypes.byref(md),
                          ctypes.byref(sv), None, None, ctypes.byref(h)) == cmx.EINVAL
    assert not h.value


def test_partition_that_cannot_hold_every_column_is_rejected():
    """A wide, thin grid has more tile columns than a few blocks of at most 64 segments can
    take: the planning query (the same partition cmx_create uses) must refuse it instead of
    leaving cells out, and accept it once there are enough blocks."""
    from paper_2603_03706_b300 import workloads as W
    p = W.make_problem(1024, 32, 1, 5e-9, W.full_mask(1024, 32, 1))   # 32 x 4 columns of 32x8
    with pytest.raises(cmx.CmxError) as ei:
        cmx.plan_tiling(p, 32, 8, 1)
    assert ei.value.code == cmx.EINVAL
    r = cmx.plan_tiling(p, 32, 8, 2)
    assert r["segments"] == 128 and r["stored"] == 1024 * 32
    with pytest.raises(cmx.CmxError):
        cmx.plan_tiling(p, 64, 4, 8)                                  # tile not compiled


def test_rows_are_stored_on_sector_boundaries():
    """Every row's stored span starts at a multiple of 8 cells, so the stored count of a sphere is
    a multiple of 8 and at least its magnetic count."""
    from paper_2603_03706_b300 import workloads as W
    for n in (8, 13, 24):
        p = W.make_problem(n, n, n, 5e-9, W.sphere_mask(n, n, n))
        r = cmx.plan_tiling(p, 32, 8, 4)
        assert r["stored"] % 8 == 0 and r["stored"] >= p.ncells, (n, r)
