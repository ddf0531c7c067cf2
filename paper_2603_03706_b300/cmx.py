"""Thin ctypes binding of libcmx (include/cmx.h): argument marshalling only.

Every step of the integration runs in the CUDA library; this module only converts arrays and
structs.  If libcmx.so is missing it raises ImportError: there is no CPU fallback.
Device arrays may be passed as torch CUDA tensors (their data pointer is used) or as plain
integers holding a device address.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcmx.so")

OK, EINVAL, ENOMEM, ECUDA, ENAN, ESTEPFAIL, ETIMEOUT, ESCRATCH, ECHECK = range(9)
MAX_MODES = 8


class CmxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"cmx status {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("cx", C.c_double),
                ("cy", C.c_double), ("cz", C.c_double), ("nsub", C.c_int)]


class Material(C.Structure):
    _fields_ = [("Ms", C.c_double), ("Aex", C.c_double), ("alpha", C.c_double),
                ("gamma", C.c_double), ("Ku", C.c_double), ("ku_axis", C.c_double * 3),
                ("B0", C.c_double * 3), ("Ndemag", C.c_double * 3), ("BE", C.c_double)]


class Modes(C.Structure):
    _fields_ = [("n_modes", C.c_int), ("omega", C.POINTER(C.c_double)),
                ("kappa", C.POINTER(C.c_double)), ("g_re", C.POINTER(C.c_double)),
                ("g_im", C.POINTER(C.c_double)), ("u", C.c_void_p), ("u_on_device", C.c_int)]


class Solver(C.Structure):
    _fields_ = [("rtol", C.c_double), ("a_ref", C.c_double), ("dt0", C.c_double),
                ("dt_min", C.c_double), ("dt_max", C.c_double), ("sample_dt", C.c_double),
                ("log_cap", C.c_int), ("trace_cap", C.c_int)]


class Tiling(C.Structure):
    _fields_ = [("bx", C.c_int), ("by", C.c_int), ("bz", C.c_int), ("blocks_per_sm", C.c_int),
                ("plain_copies", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("attempts", C.c_longlong),
                ("accepted", C.c_longlong), ("cell_stage_updates", C.c_longlong),
                ("status", C.c_int), ("launches", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Instance(C.Structure):
    _fields_ = [("grid", Grid), ("mask", C.c_void_p), ("mat", Material), ("modes", Modes),
                ("m0", C.c_void_p), ("a0", C.c_void_p), ("T", C.c_double)]


class BatchConfig(C.Structure):
    _fields_ = [("bx", C.c_int), ("by", C.c_int), ("team", C.c_int), ("blocks_per_sm", C.c_int),
                ("use_graph", C.c_int)]


class Grads(C.Structure):
    _fields_ = [("g_re", C.c_void_p), ("g_im", C.c_void_p), ("kappa", C.c_void_p),
                ("omega", C.c_void_p), ("alpha", C.c_void_p), ("a0", C.c_void_p),
                ("m0", C.c_void_p), ("m0_on_device", C.c_int), ("u", C.c_void_p),
                ("u_on_device", C.c_int), ("gb_re", C.c_void_p), ("gb_im", C.c_void_p),
                ("kerr", C.c_void_p), ("pump_re", C.c_void_p), ("pump_im", C.c_void_p)]


class Step(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("err", C.c_double),
                ("accepted", C.c_int32), ("pad", C.c_int32)]


_lib = None

# name -> (restype, argtypes); every declaration of include/cmx.h
_P = C.c_void_p
SIGNATURES = {
    "cmx_create": (C.c_int, [C.POINTER(Grid), C.c_void_p, C.POINTER(Material), C.POINTER(Modes),
                             C.POINTER(Solver), C.POINTER(Tiling), C.c_void_p, C.POINTER(C.c_void_p)]),
    "cmx_destroy": (C.c_int, [_P]),
    "cmx_set_state": (C.c_int, [_P, C.c_void_p, C.c_int, C.c_void_p, C.c_double]),
    "cmx_run": (C.c_int, [_P, C.c_double, C.c_longlong, C.POINTER(Stats)]),
    "cmx_launch": (C.c_int, [_P, C.c_double, C.c_int]),
    "cmx_replay": (C.c_int, [_P, C.c_void_p, C.c_longlong, C.POINTER(Stats)]),
    "cmx_sync": (C.c_int, [_P, C.POINTER(Stats)]),
    "cmx_eval_rhs": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cmx_get_m": (C.c_int, [_P, C.c_void_p, C.c_int]),
    "cmx_get_a": (C.c_int, [_P, C.c_void_p]),
    "cmx_get_log": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                              C.POINTER(C.c_longlong)]),
    "cmx_get_trace": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                C.POINTER(C.c_longlong)]),
    "cmx_ncells": (C.c_int, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "cmx_set_launch_attempts": (C.c_int, [_P, C.c_int]),
    "cmx_set_timeout": (C.c_int, [_P, C.c_longlong]),
    "cmx_debug_skip_arrival": (C.c_int, [_P, C.c_int]),
    "cmx_get_tiling": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "cmx_set_demag": (C.c_int, [_P, C.c_int]),
    "cmx_save_state": (C.c_int, [_P, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "cmx_load_state": (C.c_int, [_P, C.c_void_p, C.c_size_t]),
    "cmx_plan_tiling": (C.c_int, [C.POINTER(Grid), C.c_void_p, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "cmx_last_error": (C.c_char_p, [_P]),
    "cmx_checked_build": (C.c_int, []),
    "cmx_status_string": (C.c_char_p, [C.c_int]),
    "cmx_batch_create": (C.c_int, [C.POINTER(Instance), C.c_int, C.POINTER(Solver),
                                   C.POINTER(BatchConfig), C.c_void_p, C.POINTER(C.c_void_p)]),
    "cmx_batch_destroy": (C.c_int, [_P]),
    "cmx_batch_launch": (C.c_int, [_P, C.c_int]),
    "cmx_batch_run": (C.c_int, [_P, C.c_longlong, C.POINTER(Stats)]),
    "cmx_batch_stats": (C.c_int, [_P, C.c_int, C.POINTER(Stats)]),
    "cmx_batch_get_a": (C.c_int, [_P, C.c_int, C.c_void_p]),
    "cmx_batch_get_m": (C.c_int, [_P, C.c_int, C.c_void_p]),
    "cmx_batch_get_log": (C.c_int, [_P, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.POINTER(C.c_longlong)]),
    "cmx_batch_get_trace": (C.c_int, [_P, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                      C.POINTER(C.c_longlong)]),
    "cmx_batch_info": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "cmx_batch_last_error": (C.c_char_p, [_P]),
    "cmx_autotune": (C.c_int, [_P, C.c_int, C.c_void_p, C.c_void_p]),
    "cmx_set_split": (C.c_int, [_P, C.c_double]),
    "cmx_set_backward_coupling": (C.c_int, [_P, C.c_void_p, C.c_void_p]),
    "cmx_set_kerr": (C.c_int, [_P, C.c_void_p]),
    "cmx_set_pump": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cmx_set_drive": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_double, C.c_double]),
    "cmx_batch_spectrum": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                     C.c_void_p]),
    "cmx_batch_set_drive": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                      C.c_double]),
    "cmx_adjoint_record": (C.c_int, [_P, C.c_int, C.c_longlong]),
    "cmx_adjoint": (C.c_int, [_P, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Grads)]),
    "cmx_adjoint_steps": (C.c_int, [_P, C.POINTER(C.c_longlong)]),
    "cmx_batch_autotune": (C.c_int, [C.POINTER(Instance), C.c_int, C.POINTER(Solver), C.c_int,
                                     C.c_int, C.c_void_p, C.POINTER(BatchConfig), C.c_void_p,
                                     C.POINTER(C.c_int)]),
    "cmx_eval_rhs_noalloc": (C.c_int, [C.POINTER(Grid), C.c_void_p, C.POINTER(Material),
                                       C.POINTER(Modes), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
}


def load(path: Optional[str] = None):
    """Load libcmx.so (built in-tree by paper_2603_03706_b300.build); the environment variable
    CMX_LIBRARY selects another build of the same ABI (e.g. the bounds-checked libcmx_check.so)."""
    global _lib
    if _lib is None:
        p = path or os.environ.get("CMX_LIBRARY") or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} not found: build it with `python -m paper_2603_03706_b300.build`"
                              " (the integrator has no CPU fallback)")
        lib = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _dev_ptr(x) -> Optional[int]:
    """Device address of a torch CUDA tensor or an int, else None (host data)."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        return int(x.data_ptr())
    return None


def _host_f32_ptr(x) -> Optional[int]:
    """Address of a contiguous float32 torch CPU tensor (e.g. pinned memory), else None."""
    if hasattr(x, "data_ptr") and not getattr(x, "is_cuda", False):
        if str(getattr(x, "dtype", "")) == "torch.float32" and x.is_contiguous():
            return int(x.data_ptr())
    return None


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1))


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Simulation:
    """One cmx_problem handle.  Method names follow the C calls (cmx_<name>)."""

    def __init__(self, grid: Grid, mask: np.ndarray, mat: Material, omega=(), kappa=(),
                 g_re=(), g_im=(), u=None, solver: Optional[Solver] = None,
                 tiling: Optional[Tiling] = None, stream=None):
        lib = load()
        self._keep = []
        self.nsub = grid.nsub
        self.nbox = grid.nx * grid.ny * grid.nz
        self.shape = (grid.nz, grid.ny, grid.nx)
        mask = np.ascontiguousarray(np.asarray(mask, np.uint8).reshape(-1))
        if mask.size != self.nbox:
            raise ValueError("mask size")
        om, ka, gr, gi = _f64(omega), _f64(kappa), _f64(g_re), _f64(g_im)
        self.N = len(om)
        self.has_u = u is not None
        md = Modes()
        md.n_modes = self.N
        md.omega, md.kappa, md.g_re, md.g_im = _dptr(om), _dptr(ka), _dptr(gr), _dptr(gi)
        if u is None:
            md.u, md.u_on_device = None, 0
        elif _dev_ptr(u) is not None:
            md.u, md.u_on_device = _dev_ptr(u), 1
        else:
            uu = _f32(u)
            if uu.size != self.N * self.nbox:
                raise ValueError("u size")
            self._keep.append(uu)
            md.u, md.u_on_device = uu.ctypes.data, 0
        self.solver = solver or Solver(1e-6, 1e-3, 1e-13, 1e-18, 1e-11, 0.0, 0, 0)
        h = C.c_void_p()
        rc = lib.cmx_create(C.byref(grid), mask.ctypes.data, C.byref(mat), C.byref(md),
                            C.byref(self.solver), C.byref(tiling) if tiling else None,
                            _stream_handle(stream), C.byref(h))
        if rc != OK:
            raise CmxError(rc, f"cmx_create: {lib.cmx_status_string(rc).decode()}")
        self.h = h
        self._keep.clear()

    @classmethod
    def from_problem(cls, p, *, log_cap=0, trace_cap=0, sample_dt=0.0, tiling=None, stream=None,
                     u=None):
        """Build from a workloads.Problem (argument conversion only)."""
        g = Grid(p.nx, p.ny, p.nz, p.cx, p.cy, p.cz, p.nsub)
        mt = Material(p.Ms, p.Aex, p.alpha, p.gamma, p.Ku, (C.c_double * 3)(*p.ku_axis),
                      (C.c_double * 3)(*p.B0), (C.c_double * 3)(*p.Ndemag), p.BE)
        sv = Solver(p.rtol, p.a_ref, p.dt0, p.dt_min, p.dt_max, sample_dt, log_cap, trace_cap)
        tl = Tiling(*tiling) if tiling is not None else None
        sim = cls(g, p.mask, mt, p.omega, p.kappa, p.g_re, p.g_im,
                  p.u if u is None else u, sv, tl, stream)
        sim.set_state(p.m0, p.a0, 0.0)
        if getattr(p, "drive", None) is not None:
            sim.set_drive(p.drive, p.drive_t0, p.drive_sigma)
        if getattr(p, "g_back", None) is not None:
            sim.set_backward_coupling(p.g_back)
        if getattr(p, "kerr", None) is not None:
            sim.set_kerr(p.kerr)
        if getattr(p, "pump", None) is not None:
            sim.set_pump(p.pump, p.pump_omega)
        if getattr(p, "full_demag", False):
            sim.set_demag(True)
        return sim

    # -- lifetime ----------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            load().cmx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int, what: str):
        if rc != OK:
            msg = load().cmx_last_error(self.h).decode()
            raise CmxError(rc, f"{what}: {msg}")

    # -- state -------------------------------------------------------------------------------
    def set_state(self, m, a=None, t: float = 0.0):
        dp = _dev_ptr(m)
        hp = _host_f32_ptr(m)
        if dp is not None:
            mp, dev = dp, 1
        elif hp is not None:
            if m.numel() != self.nsub * 3 * self.nbox:
                raise ValueError("m size")
            mp, dev = hp, 0
        else:
            mm = _f32(m)
            if mm.size != self.nsub * 3 * self.nbox:
                raise ValueError("m size")
            mp, dev = mm.ctypes.data, 0
        aa = None
        if a is not None and self.N:
            aa = np.empty(2 * self.N)
            ac = np.asarray(a).reshape(-1)
            if np.iscomplexobj(ac):
                aa[0::2], aa[1::2] = ac.real, ac.imag
            else:
                aa[:] = ac
        self._check(load().cmx_set_state(self.h, mp, dev, aa.ctypes.data if aa is not None else None,
                                         float(t)), "set_state")

    def get_m(self, out=None):
        """Dense box magnetisation (nsub, 3, nz, ny, nx) float32; `out` may be a CUDA tensor."""
        if out is not None and _dev_ptr(out) is not None:
            self._check(load().cmx_get_m(self.h, _dev_ptr(out), 1), "get_m")
            return out
        if out is not None and _host_f32_ptr(out) is not None:
            if out.numel() != self.nsub * 3 * self.nbox:
                raise ValueError("out size")
            self._check(load().cmx_get_m(self.h, _host_f32_ptr(out), 0), "get_m")
            return out
        buf = np.empty((self.nsub, 3) + self.shape, np.float32)
        self._check(load().cmx_get_m(self.h, buf.ctypes.data, 0), "get_m")
        return buf

    def get_a(self) -> np.ndarray:
        buf = np.zeros(max(2 * self.N, 1))
        self._check(load().cmx_get_a(self.h, buf.ctypes.data), "get_a")
        return buf[0:2 * self.N:2] + 1j * buf[1:2 * self.N:2]

    # -- integration -------------------------------------------------------------------------
    def run(self, T: float, max_attempts: int = 0) -> dict:
        st = Stats()
        self._check(load().cmx_run(self.h, float(T), int(max_attempts), C.byref(st)), "run")
        return st.as_dict()

    def launch(self, T: float, n_attempts: int):
        self._check(load().cmx_launch(self.h, float(T), int(n_attempts)), "launch")

    def replay(self, dts) -> dict:
        d = _f64(dts)
        st = Stats()
        self._check(load().cmx_replay(self.h, d.ctypes.data, len(d), C.byref(st)), "replay")
        return st.as_dict()

    def sync(self) -> dict:
        st = Stats()
        self._check(load().cmx_sync(self.h, C.byref(st)), "sync")
        return st.as_dict()

    def status(self) -> int:
        st = Stats()
        return load().cmx_sync(self.h, C.byref(st))

    def eval_rhs(self, m, a=None):
        """f(m, a): (dm dense float32, da complex, <m^-> complex)."""
        mm = _f32(m)
        dm = np.empty((self.nsub, 3) + self.shape, np.float32)
        aa = np.zeros(max(2 * self.N, 1))
        if a is not None and self.N:
            ac = np.asarray(a).reshape(-1)
            aa[0:2 * self.N:2], aa[1:2 * self.N:2] = ac.real, ac.imag
        da = np.zeros(max(2 * self.N, 1))
        mo = np.zeros(max(2 * self.N, 1))
        self._check(load().cmx_eval_rhs(self.h, mm.ctypes.data, aa.ctypes.data, dm.ctypes.data,
                                        da.ctypes.data, mo.ctypes.data), "eval_rhs")
        cx = lambda v: v[0:2 * self.N:2] + 1j * v[1:2 * self.N:2]
        return dm, cx(da), cx(mo)

    # -- records -----------------------------------------------------------------------------
    def get_log(self, cap: Optional[int] = None) -> dict:
        cap = self.solver.log_cap if cap is None else cap
        steps = (Step * max(cap, 1))()
        Q = max(2 * self.N, 1)
        a = np.zeros(max(cap, 1) * Q)
        mm = np.zeros(max(cap, 1) * Q)
        n = C.c_longlong()
        self._check(load().cmx_get_log(self.h, steps, a.ctypes.data, mm.ctypes.data, cap,
                                       C.byref(n)), "get_log")
        k = min(cap, n.value)
        arr = np.ctypeslib.as_array(steps)[:k] if k else None
        out = dict(n=n.value,
                   t=np.array([s.t for s in steps[:k]]), dt=np.array([s.dt for s in steps[:k]]),
                   err=np.array([s.err for s in steps[:k]]),
                   accepted=np.array([bool(s.accepted) for s in steps[:k]], bool))
        del arr
        if self.N:
            a = a[:k * 2 * self.N]
            mm = mm[:k * 2 * self.N]
            out["a"] = (a[0::2] + 1j * a[1::2]).reshape(k, self.N)
            out["mm"] = (mm[0::2] + 1j * mm[1::2]).reshape(k, self.N)
        return out

    def get_trace(self, cap: Optional[int] = None) -> dict:
        cap = self.solver.trace_cap if cap is None else cap
        Q = max(2 * self.N, 1)
        t = np.zeros(max(cap, 1))
        a = np.zeros(max(cap, 1) * Q)
        mm = np.zeros(max(cap, 1) * Q)
        n = C.c_longlong()
        self._check(load().cmx_get_trace(self.h, t.ctypes.data, a.ctypes.data, mm.ctypes.data, cap,
                                         C.byref(n)), "get_trace")
        k = min(cap, n.value)
        out = dict(n=n.value, t=t[:k])
        if self.N:
            a, mm = a[:k * 2 * self.N], mm[:k * 2 * self.N]
            out["a"] = (a[0::2] + 1j * a[1::2]).reshape(k, self.N)
            out["mm"] = (mm[0::2] + 1j * mm[1::2]).reshape(k, self.N)
        return out

    # -- adjoint -----------------------------------------------------------------------------
    def adjoint_record(self, every: int, max_steps: int):
        """Arm the checkpoint store for the next run (right after set_state)."""
        self._check(load().cmx_adjoint_record(self.h, int(every), int(max_steps)),
                    "adjoint_record")

    def adjoint_steps(self) -> int:
        n = C.c_longlong()
        self._check(load().cmx_adjoint_steps(self.h, C.byref(n)), "adjoint_steps")
        return n.value

    def adjoint(self, dL_da=None, dL_dm=None, want_u: bool = True, want_m0: bool = True) -> dict:
        """Gradients of a loss through the recorded run (cmx_adjoint).

        dL_da: (n+1, N) complex or (n+1, 2N) packed reals, dL/d a_i for the states after i
        accepted steps; dL_dm: dense (nsub, 3, nz, ny, nx) FP32 or None.  Returns numpy arrays:
        g_re, g_im, kappa, omega (N), alpha (float), a0 (N complex: dL/dRe + i dL/dIm), m0 (dense)
        and u ((N, nz, ny, nx) float64, with mode profiles).
        """
        N = self.N
        n = self.adjoint_steps()
        la = None
        if dL_da is not None:
            d = np.asarray(dL_da)
            if np.iscomplexobj(d):
                d = np.stack([d.real, d.imag], -1)
            la = _f64(d)
            if la.size != (n + 1) * 2 * N:
                raise ValueError(f"dL_da must hold {n + 1} x {2 * N} values")
        lm = None if dL_dm is None else _f32(dL_dm)
        if lm is not None and lm.size != 3 * self.nsub * self.nbox:
            raise ValueError("dL_dm size")
        out = {k: np.zeros(max(N, 1))
               for k in ("g_re", "g_im", "kappa", "omega", "gb_re", "gb_im", "kerr", "pump_re",
                         "pump_im")}
        alpha = np.zeros(1)
        a0 = np.zeros(max(2 * N, 1))
        m0 = np.zeros(3 * self.nsub * self.nbox, np.float32) if want_m0 else None
        u = np.zeros(max(N, 1) * self.nbox) if (want_u and self.has_u) else None
        g = Grads(out["g_re"].ctypes.data, out["g_im"].ctypes.data, out["kappa"].ctypes.data,
                  out["omega"].ctypes.data, alpha.ctypes.data, a0.ctypes.data,
                  m0.ctypes.data if m0 is not None else None, 0,
                  u.ctypes.data if u is not None else None, 0, out["gb_re"].ctypes.data,
                  out["gb_im"].ctypes.data, out["kerr"].ctypes.data,
                  out["pump_re"].ctypes.data, out["pump_im"].ctypes.data)
        self._check(load().cmx_adjoint(self.h, la.ctypes.data if la is not None else None,
                                       lm.ctypes.data if lm is not None else None, 0,
                                       C.byref(g)), "adjoint")
        res = {k: v[:N].copy() for k, v in out.items()}
        res["alpha"] = float(alpha[0])
        res["a0"] = a0[0:2 * N:2] + 1j * a0[1:2 * N:2]
        res["a0_packed"] = a0[:2 * N].copy()
        res["n"] = n
        if m0 is not None:
            res["m0"] = m0.reshape((self.nsub, 3) + self.shape)
        if u is not None:
            res["u"] = u[:N * self.nbox].reshape((N,) + self.shape)
        return res

    # -- configuration -----------------------------------------------------------------------
    def ncells(self):
        a, b = C.c_longlong(), C.c_longlong()
        self._check(load().cmx_ncells(self.h, C.byref(a), C.byref(b)), "ncells")
        return a.value, b.value

    def set_launch_attempts(self, n: int):
        self._check(load().cmx_set_launch_attempts(self.h, int(n)), "set_launch_attempts")

    def set_timeout(self, ns: int):
        self._check(load().cmx_set_timeout(self.h, int(ns)), "set_timeout")

    def debug_skip_arrival(self, block: int):
        self._check(load().cmx_debug_skip_arrival(self.h, int(block)), "debug_skip_arrival")

    def set_split(self, ds: float):
        """cmx_set_split: operator-split scheme with interval ds (0: the coupled scheme)."""
        self._check(load().cmx_set_split(self.h, float(ds)), "set_split")

    def save_state(self) -> bytes:
        """cmx_save_state: the integrator's state as a host blob."""
        n = C.c_size_t()
        self._check(load().cmx_save_state(self.h, None, 0, C.byref(n)), "save_state")
        buf = (C.c_ubyte * n.value)()
        self._check(load().cmx_save_state(self.h, buf, n.value, None), "save_state")
        return bytes(buf)

    def load_state(self, blob: bytes):
        """cmx_load_state: resume from a blob of save_state (same problem and settings)."""
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        self._check(load().cmx_load_state(self.h, buf, len(blob)), "load_state")

    def set_demag(self, full: bool):
        """cmx_set_demag: full magnetostatic demag (True) or the diagonal factors (False)."""
        self._check(load().cmx_set_demag(self.h, 1 if full else 0), "set_demag")

    def set_backward_coupling(self, gb=None):
        """cmx_set_backward_coupling: complex backward coefficients gb~_n of the feedback field
        (nonreciprocal coupling); None restores reciprocal coupling."""
        if gb is None:
            self._check(load().cmx_set_backward_coupling(self.h, None, None), "backward_coupling")
            return
        g = np.asarray(gb, complex).reshape(-1)
        if g.size != self.N:
            raise ValueError("one backward coefficient per mode")
        re, im = _f64(g.real), _f64(g.imag)
        self._check(load().cmx_set_backward_coupling(self.h, re.ctypes.data, im.ctypes.data),
                    "backward_coupling")

    def set_kerr(self, kerr=None):
        """cmx_set_kerr: self-Kerr coefficients K_n (None: no Kerr term)."""
        if kerr is None:
            self._check(load().cmx_set_kerr(self.h, None), "set_kerr")
            return
        k = _f64(kerr)
        if k.size != self.N:
            raise ValueError("one Kerr coefficient per mode")
        self._check(load().cmx_set_kerr(self.h, k.ctypes.data), "set_kerr")

    def set_pump(self, pump=None, omega_p=None):
        """cmx_set_pump: degenerate parametric pump -i P_n e^{-i wp_n t} conj(a_n) on da_n/dt
        (pump: N complex P_n [rad/s], omega_p: N pump frequencies [rad/s]; None: no pump)."""
        if pump is None:
            self._check(load().cmx_set_pump(self.h, None, None, None), "set_pump")
            return
        P = np.asarray(pump, complex).reshape(-1)
        wp = _f64(omega_p)
        if P.size != self.N or wp.size != self.N:
            raise ValueError("one pump coefficient and frequency per mode")
        re, im = _f64(P.real), _f64(P.imag)
        self._check(load().cmx_set_pump(self.h, re.ctypes.data, im.ctypes.data, wp.ctypes.data),
                    "set_pump")

    def set_drive(self, eta=None, t0: float = 0.1e-9, sigma: float = 20e-12):
        """cmx_set_drive: Gaussian drive eta_n exp(-(t-t0)^2/(2 sigma^2)) on da_n/dt
        (eta: N complex amplitudes [1/s]; None switches it off)."""
        if eta is None:
            self._check(load().cmx_set_drive(self.h, None, None, 0.0, 1.0), "set_drive")
            return
        e = np.asarray(eta, complex).reshape(-1)
        if e.size != self.N:
            raise ValueError("one drive amplitude per mode")
        re, im = _f64(e.real), _f64(e.imag)
        self._check(load().cmx_set_drive(self.h, re.ctypes.data, im.ctypes.data, float(t0),
                                         float(sigma)), "set_drive")

    def autotune(self, attempts: int = 20) -> dict:
        """cmx_autotune: time the compiled tiles (and, for a small grid, the single-block
        integrator) from the current state, keep the fastest (bx = by = 0: single block)."""
        t = Tiling()
        us = np.zeros(4)
        self._check(load().cmx_autotune(self.h, int(attempts), C.byref(t), us.ctypes.data),
                    "autotune")
        return dict(bx=t.bx, by=t.by, bz=t.bz, us_per_attempt=dict(
            zip(("32x4", "32x8", "32x16", "single_block"), [float(v) for v in us])))

    def get_tiling(self) -> dict:
        v = [C.c_int() for _ in range(6)]
        self._check(load().cmx_get_tiling(self.h, *[C.byref(x) for x in v]), "get_tiling")
        return dict(zip(("bx", "by", "bz", "blocks", "tiles", "dense"), [x.value for x in v]))

    def last_error(self) -> str:
        return load().cmx_last_error(self.h).decode()


def _unpack_complex(v, N):
    return v[0:2 * N:2] + 1j * v[1:2 * N:2]


def _instances(problems):
    """cmx_instance array for a list of workloads.Problem (argument conversion only); returns
    (array, arrays to keep alive, modes per instance, shapes)."""
    keep = []
    n = len(problems)
    arr = (Instance * n)()
    Ns, shapes = [], []
    for i, p in enumerate(problems):
        if p.u is not None:
            raise ValueError("batched problems use uniform mode profiles (u = None)")
        mask = np.ascontiguousarray(np.asarray(p.mask, np.uint8).reshape(-1))
        om, ka, gr, gi = _f64(p.omega), _f64(p.kappa), _f64(p.g_re), _f64(p.g_im)
        m0 = _f32(p.m0)
        a0 = np.zeros(max(2 * p.nmodes, 1))
        if p.nmodes:
            ac = np.asarray(p.a0, complex).reshape(-1)
            a0[0:2 * p.nmodes:2], a0[1:2 * p.nmodes:2] = ac.real, ac.imag
        keep += [mask, om, ka, gr, gi, m0, a0]
        ins = arr[i]
        ins.grid = Grid(p.nx, p.ny, p.nz, p.cx, p.cy, p.cz, p.nsub)
        ins.mask = mask.ctypes.data
        ins.mat = Material(p.Ms, p.Aex, p.alpha, p.gamma, p.Ku, (C.c_double * 3)(*p.ku_axis),
                           (C.c_double * 3)(*p.B0), (C.c_double * 3)(*p.Ndemag), p.BE)
        md = Modes()
        md.n_modes = p.nmodes
        md.omega, md.kappa, md.g_re, md.g_im = _dptr(om), _dptr(ka), _dptr(gr), _dptr(gi)
        md.u, md.u_on_device = None, 0
        ins.modes = md
        ins.m0 = m0.ctypes.data
        ins.a0 = a0.ctypes.data
        ins.T = p.T
        Ns.append(p.nmodes)
        shapes.append((p.nz, p.ny, p.nx))
    return arr, keep, Ns, shapes


def batch_autotune(problems, *, sample=64, attempts=20, blocks_per_sm=0, use_graph=True,
                   stream=None) -> dict:
    """cmx_batch_autotune: time the candidate launch shapes on trial batches of every k-th
    problem and return the fastest (bx, by, team) with the times of all candidates."""
    arr, keep, _, _ = _instances(problems)
    p0 = problems[0]
    sv = Solver(p0.rtol, p0.a_ref, p0.dt0, p0.dt_min, p0.dt_max, 0.0, 0, 0)
    cfg = BatchConfig(0, 0, 0, blocks_per_sm, 1 if use_graph else 0)
    us = np.full(12, np.nan)
    nc = C.c_int()
    rc = load().cmx_batch_autotune(arr, len(problems), C.byref(sv), int(sample), int(attempts),
                                   _stream_handle(stream), C.byref(cfg), us.ctypes.data,
                                   C.byref(nc))
    if rc != OK:
        raise CmxError(rc, f"cmx_batch_autotune: {load().cmx_status_string(rc).decode()}")
    del keep
    return dict(bx=cfg.bx, by=cfg.by, team=cfg.team, us=us[:nc.value].tolist())


class BatchSimulation:
    """One cmx_batch handle (cmx_batch_* calls): independent problems in one persistent launch."""

    def __init__(self, problems, *, log_cap=0, trace_cap=0, sample_dt=0.0, solver=None,
                 bx=0, by=0, team=0, blocks_per_sm=0, use_graph=True, stream=None):
        lib = load()
        n = len(problems)
        arr, keep, self.N, self.shapes = _instances(problems)
        self.nsub = problems[0].nsub
        p0 = problems[0]
        self.solver = solver or Solver(p0.rtol, p0.a_ref, p0.dt0, p0.dt_min, p0.dt_max, sample_dt,
                                       log_cap, trace_cap)
        cfg = BatchConfig(bx, by, team, blocks_per_sm, 1 if use_graph else 0)
        h = C.c_void_p()
        rc = lib.cmx_batch_create(arr, n, C.byref(self.solver), C.byref(cfg),
                                  _stream_handle(stream), C.byref(h))
        if rc != OK:
            raise CmxError(rc, f"cmx_batch_create: {lib.cmx_status_string(rc).decode()}")
        self.h = h
        self.n = n
        if getattr(p0, "drive", None) is not None:
            self.set_drive(p0.drive, p0.drive_t0, p0.drive_sigma)

    def spectrum(self, mode: int, f0: float, df: float, nf: int, t_start: float = 0.0):
        """cmx_batch_spectrum: |windowed DFT|^2 of every instance's trace of a_mode at
        f0 + j df (Hz); returns an (n, nf) array."""
        out = np.zeros(self.n * int(nf))
        self._check(load().cmx_batch_spectrum(self.h, int(mode), float(f0), float(df), int(nf),
                                              float(t_start), out.ctypes.data), "batch_spectrum")
        return out.reshape(self.n, int(nf))

    def set_drive(self, eta=None, t0: float = 0.1e-9, sigma: float = 20e-12):
        """cmx_batch_set_drive: the same Gaussian drive for every instance (eta: amplitudes
        of modes 0.. [1/s]; None switches it off)."""
        lib = load()
        if eta is None:
            rc = lib.cmx_batch_set_drive(self.h, None, None, 0, 0.0, 1.0)
        else:
            e = np.asarray(eta, complex).reshape(-1)
            re, im = _f64(e.real), _f64(e.imag)
            rc = lib.cmx_batch_set_drive(self.h, re.ctypes.data, im.ctypes.data, e.size,
                                         float(t0), float(sigma))
        self._check(rc, "batch_set_drive")

    def close(self):
        if getattr(self, "h", None):
            load().cmx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != OK:
            raise CmxError(rc, f"{what}: {load().cmx_batch_last_error(self.h).decode()}")

    def launch(self, n_attempts: int):
        self._check(load().cmx_batch_launch(self.h, int(n_attempts)), "batch_launch")

    def run(self, max_attempts: int = 0) -> dict:
        st = Stats()
        self._check(load().cmx_batch_run(self.h, int(max_attempts), C.byref(st)), "batch_run")
        return st.as_dict()

    def stats(self, i: int) -> dict:
        st = Stats()
        self._check(load().cmx_batch_stats(self.h, int(i), C.byref(st)), "batch_stats")
        return st.as_dict()

    def get_a(self, i: int) -> np.ndarray:
        buf = np.zeros(max(2 * self.N[i], 1))
        self._check(load().cmx_batch_get_a(self.h, int(i), buf.ctypes.data), "batch_get_a")
        return _unpack_complex(buf, self.N[i])

    def get_m(self, i: int) -> np.ndarray:
        buf = np.empty((self.nsub, 3) + self.shapes[i], np.float32)
        self._check(load().cmx_batch_get_m(self.h, int(i), buf.ctypes.data), "batch_get_m")
        return buf

    def get_log(self, i: int, cap=None) -> dict:
        cap = self.solver.log_cap if cap is None else cap
        N = self.N[i]
        steps = (Step * max(cap, 1))()
        Q = max(2 * N, 1)
        a = np.zeros(max(cap, 1) * Q)
        mm = np.zeros(max(cap, 1) * Q)
        n = C.c_longlong()
        self._check(load().cmx_batch_get_log(self.h, int(i), steps, a.ctypes.data, mm.ctypes.data,
                                             cap, C.byref(n)), "batch_get_log")
        k = min(cap, n.value)
        out = dict(n=n.value, t=np.array([s.t for s in steps[:k]]),
                   dt=np.array([s.dt for s in steps[:k]]),
                   err=np.array([s.err for s in steps[:k]]),
                   accepted=np.array([bool(s.accepted) for s in steps[:k]], bool))
        if N:
            out["a"] = (a[:k * 2 * N][0::2] + 1j * a[:k * 2 * N][1::2]).reshape(k, N)
            out["mm"] = (mm[:k * 2 * N][0::2] + 1j * mm[:k * 2 * N][1::2]).reshape(k, N)
        return out

    def get_trace(self, i: int, cap=None) -> dict:
        cap = self.solver.trace_cap if cap is None else cap
        N = self.N[i]
        Q = max(2 * N, 1)
        t = np.zeros(max(cap, 1))
        a = np.zeros(max(cap, 1) * Q)
        mm = np.zeros(max(cap, 1) * Q)
        n = C.c_longlong()
        self._check(load().cmx_batch_get_trace(self.h, int(i), t.ctypes.data, a.ctypes.data,
                                               mm.ctypes.data, cap, C.byref(n)), "batch_get_trace")
        k = min(cap, n.value)
        out = dict(n=n.value, t=t[:k])
        if N:
            out["a"] = (a[:k * 2 * N][0::2] + 1j * a[:k * 2 * N][1::2]).reshape(k, N)
            out["mm"] = (mm[:k * 2 * N][0::2] + 1j * mm[:k * 2 * N][1::2]).reshape(k, N)
        return out

    def info(self) -> dict:
        v = [C.c_int(), C.c_int(), C.c_int(), C.c_longlong(), C.c_int()]
        self._check(load().cmx_batch_info(self.h, *[C.byref(x) for x in v]), "batch_info")
        return dict(zip(("teams", "team_size", "blocks", "cells", "graph"), [x.value for x in v]))


def plan_tiling(p, bx: int, by: int, blocks: int) -> dict:
    """cmx_plan_tiling (host only): segments and stored cells of the partition of workloads
    Problem p into `blocks` blocks of bx x by tiles; raises CmxError when it does not fit."""
    g = Grid(p.nx, p.ny, p.nz, p.cx, p.cy, p.cz, p.nsub)
    mask = np.ascontiguousarray(np.asarray(p.mask, np.uint8).reshape(-1))
    nseg, nst = C.c_longlong(), C.c_longlong()
    rc = load().cmx_plan_tiling(C.byref(g), mask.ctypes.data, int(bx), int(by), int(blocks),
                                C.byref(nseg), C.byref(nst))
    if rc != OK:
        raise CmxError(rc, "cmx_plan_tiling: " + load().cmx_status_string(rc).decode())
    return dict(segments=nseg.value, stored=nst.value)


def eval_rhs_noalloc(p, m_dev, dm_dev, a=None, stream=None, u_dev=None):
    """cmx_eval_rhs_noalloc for a workloads.Problem: m_dev, dm_dev are device pointers (or CUDA
    tensors) of dense-box float32 arrays; u_dev (optional) a device pointer or CUDA tensor of the
    dense-box profiles, used instead of the host copy p.u.  Returns (da, mm) complex; raises
    CmxError."""
    lib = load()
    g = Grid(p.nx, p.ny, p.nz, p.cx, p.cy, p.cz, p.nsub)
    mt = Material(p.Ms, p.Aex, p.alpha, p.gamma, p.Ku, (C.c_double * 3)(*p.ku_axis),
                  (C.c_double * 3)(*p.B0), (C.c_double * 3)(*p.Ndemag), p.BE)
    mask = np.ascontiguousarray(np.asarray(p.mask, np.uint8).reshape(-1))
    om, ka, gr, gi = _f64(p.omega), _f64(p.kappa), _f64(p.g_re), _f64(p.g_im)
    md = Modes()
    md.n_modes = p.nmodes
    md.omega, md.kappa, md.g_re, md.g_im = _dptr(om), _dptr(ka), _dptr(gr), _dptr(gi)
    uu = None
    if u_dev is not None:
        md.u, md.u_on_device = _dev_ptr(u_dev), 1
    elif p.u is not None:
        uu = _f32(p.u)
        md.u, md.u_on_device = uu.ctypes.data, 0
    else:
        md.u, md.u_on_device = None, 0
    N = p.nmodes
    aa = np.zeros(max(2 * N, 1))
    if a is not None and N:
        ac = np.asarray(a).reshape(-1)
        aa[0:2 * N:2], aa[1:2 * N:2] = ac.real, ac.imag
    da = np.zeros(max(2 * N, 1))
    mm = np.zeros(max(2 * N, 1))
    rc = lib.cmx_eval_rhs_noalloc(C.byref(g), mask.ctypes.data, C.byref(mt), C.byref(md),
                                  _dev_ptr(m_dev), aa.ctypes.data, _dev_ptr(dm_dev),
                                  da.ctypes.data, mm.ctypes.data, _stream_handle(stream))
    if rc != OK:
        raise CmxError(rc, "cmx_eval_rhs_noalloc: " + lib.cmx_status_string(rc).decode())
    return _unpack_complex(da, N), _unpack_complex(mm, N)
