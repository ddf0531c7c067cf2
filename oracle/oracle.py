"""Python handle on the FP64 CPU oracle (``cmx_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the benchmark
may use this module; the product path never does.  It shares no code with the CUDA path; the
only thing both sides see is the input description produced by the seeded generators.

Functions
---------
``OracleProblem(problem)``   packs a workloads.Problem into the C struct (all FP64).
``rhs(op, m, a)``            f(m, a): slopes dm/dt, da/dt and the overlaps <m^->_n (Eq. (18)).
``Integrator(op)``           adaptive Dormand-Prince 5(4) run to T, or replay of given steps.
``jacobian(op, m, a)``       central-difference Jacobian of the right-hand side (for the
                             linearised-eigenvalue pins, Sec. II B, F, G).
``tableau()``                the oracle's own Butcher tableau (for the order-condition pin).
``Integrator.run_split``     the operator-split scheme of the paper's Python tier (comparison).
``rhs_vjp(op, m, a, wm, wa)`` transposed derivative of f applied to adjoint weights, with the
                             parameter gradients (g~_n, kappa_n, omega_n, alpha, u_n(r)).
``adjoint(op, m0, a0, dts, dL_da, dL_dm)``  gradient of a loss on the states a_0..a_n and m_n
                             through n replayed steps (discrete adjoint, step sizes fixed).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cmx_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ENAN, ORC_ESTEPFAIL = 0, 1, 2, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP over the cell loop, no fast-math)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC,
                               "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("nsub", C.c_int),
                ("nmodes", C.c_int), ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
                ("mask", C.POINTER(C.c_uint8)), ("Ms", C.c_double), ("Aex", C.c_double),
                ("alpha", C.c_double), ("gamma", C.c_double), ("Ku", C.c_double),
                ("ku", C.c_double * 3), ("B0", C.c_double * 3), ("Nd", C.c_double * 3),
                ("BE", C.c_double), ("u", C.POINTER(C.c_double)),
                ("omega", C.POINTER(C.c_double)), ("kappa", C.POINTER(C.c_double)),
                ("g_re", C.POINTER(C.c_double)), ("g_im", C.POINTER(C.c_double)),
                ("drive_re", C.POINTER(C.c_double)), ("drive_im", C.POINTER(C.c_double)),
                ("drive_t0", C.c_double), ("drive_sigma", C.c_double),
                ("gb_re", C.POINTER(C.c_double)), ("gb_im", C.POINTER(C.c_double)),
                ("kerr", C.POINTER(C.c_double)), ("cavity_frozen", C.c_int),
                ("pump_re", C.POINTER(C.c_double)), ("pump_im", C.POINTER(C.c_double)),
                ("pump_w", C.POINTER(C.c_double)),
                ("demag", C.POINTER(C.c_double))]


class _Solver(C.Structure):
    _fields_ = [("rtol", C.c_double), ("a_ref", C.c_double), ("dt_min", C.c_double),
                ("dt_max", C.c_double)]


class _Log(C.Structure):
    _fields_ = [("cap", C.c_int), ("n", C.c_int), ("t", C.POINTER(C.c_double)),
                ("dt", C.POINTER(C.c_double)), ("err", C.POINTER(C.c_double)),
                ("accepted", C.POINTER(C.c_int)), ("a", C.POINTER(C.c_double)),
                ("mm", C.POINTER(C.c_double))]


class _Grads(C.Structure):
    _fields_ = [("g_re", C.POINTER(C.c_double)), ("g_im", C.POINTER(C.c_double)),
                ("kappa", C.POINTER(C.c_double)), ("omega", C.POINTER(C.c_double)),
                ("alpha", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)),
                ("gb_re", C.POINTER(C.c_double)), ("gb_im", C.POINTER(C.c_double)),
                ("kerr", C.POINTER(C.c_double)), ("pump_re", C.POINTER(C.c_double)),
                ("pump_im", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER(_Problem)
        vp = C.c_void_p
        dp = C.POINTER(C.c_double)
        _lib.orc_rhs.argtypes = [P, dp, dp, dp, dp, dp]
        _lib.orc_rhs.restype = C.c_int
        _lib.orc_overlap.argtypes = [P, dp, dp]
        _lib.orc_state_new.argtypes = [P]
        _lib.orc_state_new.restype = vp
        _lib.orc_state_free.argtypes = [vp]
        _lib.orc_state_set.argtypes = [vp, dp, dp, C.c_double, C.c_double]
        _lib.orc_state_get.argtypes = [vp, dp, dp, dp, dp, C.POINTER(C.c_long)]
        _lib.orc_run.argtypes = [P, vp, C.POINTER(_Solver), C.c_double, C.c_long,
                                 C.POINTER(_Log)]
        _lib.orc_run.restype = C.c_int
        _lib.orc_replay.argtypes = [P, vp, C.POINTER(_Solver), dp, C.c_long, C.POINTER(_Log)]
        _lib.orc_replay.restype = C.c_int
        _lib.orc_run_split.argtypes = [P, vp, C.POINTER(_Solver), C.c_double, C.c_double,
                                       C.c_long, C.POINTER(_Log)]
        _lib.orc_run_split.restype = C.c_int
        _lib.orc_tableau.argtypes = [dp, dp, dp]
        _lib.orc_demag_tensor.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                          C.c_double, dp]
        _lib.orc_demag_field.argtypes = [P, dp, dp]
        _lib.orc_demag_field.restype = C.c_int
        G = C.POINTER(_Grads)
        _lib.orc_rhs_vjp.argtypes = [P, dp, dp, dp, dp, dp, dp, G]
        _lib.orc_rhs_vjp.restype = C.c_int
        _lib.orc_adjoint.argtypes = [P, C.POINTER(_Solver), dp, dp, dp, C.c_long, dp, dp, dp,
                                     dp, G, C.c_double]
        _lib.orc_adjoint.restype = C.c_int
    return _lib


def _dptr(x: np.ndarray):
    return x.ctypes.data_as(C.POINTER(C.c_double))


class OracleProblem:
    """FP64 copy of a workloads.Problem in the oracle's C struct (keeps its arrays alive)."""

    def __init__(self, p):
        self.p = p
        self.nbox = p.nx * p.ny * p.nz
        self.N = p.nmodes
        self.mask = np.ascontiguousarray(p.mask.reshape(-1), dtype=np.uint8)
        self.u = None if p.u is None else np.ascontiguousarray(
            np.asarray(p.u, np.float64).reshape(self.N, -1))
        arr = lambda v: np.ascontiguousarray(np.asarray(v, np.float64).reshape(-1))
        self.omega, self.kappa = arr(p.omega), arr(p.kappa)
        self.g_re, self.g_im = arr(p.g_re), arr(p.g_im)
        s = _Problem()
        s.nx, s.ny, s.nz, s.nsub, s.nmodes = p.nx, p.ny, p.nz, p.nsub, self.N
        s.cx, s.cy, s.cz = p.cx, p.cy, p.cz
        s.mask = self.mask.ctypes.data_as(C.POINTER(C.c_uint8))
        s.Ms, s.Aex, s.alpha, s.gamma, s.Ku = p.Ms, p.Aex, p.alpha, p.gamma, p.Ku
        s.ku[:] = list(map(float, p.ku_axis))
        s.B0[:] = list(map(float, p.B0))
        s.Nd[:] = list(map(float, p.Ndemag))
        s.BE = p.BE
        s.u = _dptr(self.u) if self.u is not None else C.POINTER(C.c_double)()
        s.omega, s.kappa = _dptr(self.omega), _dptr(self.kappa)
        s.g_re, s.g_im = _dptr(self.g_re), _dptr(self.g_im)
        drive = getattr(p, "drive", None)
        if drive is not None:
            d = np.asarray(drive, complex).reshape(-1)
            self.drive_re = np.ascontiguousarray(d.real, np.float64)
            self.drive_im = np.ascontiguousarray(d.imag, np.float64)
            s.drive_re, s.drive_im = _dptr(self.drive_re), _dptr(self.drive_im)
            s.drive_t0, s.drive_sigma = p.drive_t0, p.drive_sigma
        else:
            s.drive_re = s.drive_im = C.POINTER(C.c_double)()
            s.drive_t0, s.drive_sigma = 0.0, 1.0
        gb = getattr(p, "g_back", None)
        if gb is not None:
            g = np.asarray(gb, complex).reshape(-1)
            self.gb_re = np.ascontiguousarray(g.real, np.float64)
            self.gb_im = np.ascontiguousarray(g.imag, np.float64)
            s.gb_re, s.gb_im = _dptr(self.gb_re), _dptr(self.gb_im)
        else:
            s.gb_re = s.gb_im = C.POINTER(C.c_double)()
        kerr = getattr(p, "kerr", None)
        if kerr is not None:
            self.kerr = np.ascontiguousarray(np.asarray(kerr, np.float64).reshape(-1))
            s.kerr = _dptr(self.kerr)
        else:
            s.kerr = C.POINTER(C.c_double)()
        pump = getattr(p, "pump", None)
        if pump is not None:
            P = np.asarray(pump, complex).reshape(-1)
            self.pump_re = np.ascontiguousarray(P.real, np.float64)
            self.pump_im = np.ascontiguousarray(P.imag, np.float64)
            self.pump_w = np.ascontiguousarray(np.asarray(p.pump_omega, np.float64).reshape(-1))
            s.pump_re, s.pump_im = _dptr(self.pump_re), _dptr(self.pump_im)
            s.pump_w = _dptr(self.pump_w)
        else:
            s.pump_re = s.pump_im = s.pump_w = C.POINTER(C.c_double)()
        if getattr(p, "full_demag", False):
            self.demag = demag_tensor(p.nx, p.ny, p.nz, p.cx, p.cy, p.cz)
            s.demag = _dptr(self.demag)
        else:
            s.demag = C.POINTER(C.c_double)()
        self.s = s
        self.solver = _Solver(p.rtol, p.a_ref, p.dt_min, p.dt_max)

    @property
    def ref(self):
        return C.byref(self.s)

    def m0(self) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(self.p.m0, np.float64).reshape(-1))

    def a0(self) -> np.ndarray:
        return pack_a(self.p.a0)


def demag_tensor(nx, ny, nz, cx, cy, cz) -> np.ndarray:
    """Cell-pair demag tensor (Newell, Williams & Dunlop 1993) of every displacement of an
    nx x ny x nz grid of cx x cy x cz cells: array (6, 2nz-1, 2ny-1, 2nx-1), components
    xx, yy, zz, xy, xz, yz, index [c, k + nz-1, j + ny-1, i + nx-1] for displacement
    (i cx, j cy, k cz)."""
    out = np.empty(6 * (2 * nx - 1) * (2 * ny - 1) * (2 * nz - 1))
    lib().orc_demag_tensor(int(nx), int(ny), int(nz), float(cx), float(cy), float(cz),
                           _dptr(out))
    return out.reshape(6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1)


def demag_field(op: OracleProblem, m: np.ndarray) -> np.ndarray:
    """Full demag field (T) of state m (flat FP64, nsub*3*nbox) at every cell: (3, nbox)."""
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    out = np.empty(3 * op.nbox)
    rc = lib().orc_demag_field(op.ref, _dptr(m), _dptr(out))
    if rc:
        raise RuntimeError("orc_demag_field: the problem has no full demag")
    return out.reshape(3, op.nbox)


def pack_a(a) -> np.ndarray:
    a = np.asarray(a, complex).reshape(-1)
    out = np.empty(2 * len(a))
    out[0::2], out[1::2] = a.real, a.imag
    return out


def unpack_a(x) -> np.ndarray:
    x = np.asarray(x, float).reshape(-1)
    return x[0::2] + 1j * x[1::2]


def rhs(op: OracleProblem, m: np.ndarray, a: np.ndarray):
    """Slopes (dm, da) and overlaps mm at (m, a); m flat FP64 (nsub*3*nbox), a packed (2N)."""
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    a = np.ascontiguousarray(a, np.float64).reshape(-1)
    dm = np.empty_like(m)
    da = np.empty(max(2 * op.N, 1))
    mm = np.empty(max(2 * op.N, 1))
    rc = lib().orc_rhs(op.ref, _dptr(m), _dptr(a), _dptr(dm), _dptr(da), _dptr(mm))
    if rc:
        raise RuntimeError(f"orc_rhs failed: {rc}")
    return dm, da[:2 * op.N], mm[:2 * op.N]


def overlap(op: OracleProblem, m: np.ndarray) -> np.ndarray:
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    mm = np.empty(max(2 * op.N, 1))
    lib().orc_overlap(op.ref, _dptr(m), _dptr(mm))
    return unpack_a(mm[:2 * op.N])


def tableau():
    a = np.zeros((7, 6))
    b5 = np.zeros(7)
    b4 = np.zeros(7)
    lib().orc_tableau(_dptr(a), _dptr(b5), _dptr(b4))
    return a, b5, b4


class Log:
    """Per-attempt record: t, dt, err, accepted, a (complex, N) and <m^-> at the stage-7 point."""

    def __init__(self, cap: int, N: int):
        self.cap, self.N = cap, N
        self.t = np.zeros(cap)
        self.dt = np.zeros(cap)
        self.err = np.zeros(cap)
        self.accepted = np.zeros(cap, np.int32)
        self.a = np.zeros(cap * max(2 * N, 1))
        self.mm = np.zeros(cap * max(2 * N, 1))
        s = _Log()
        s.cap, s.n = cap, 0
        s.t, s.dt, s.err = _dptr(self.t), _dptr(self.dt), _dptr(self.err)
        s.accepted = self.accepted.ctypes.data_as(C.POINTER(C.c_int))
        s.a, s.mm = _dptr(self.a), _dptr(self.mm)
        self.s = s

    @property
    def n(self) -> int:
        return min(self.s.n, self.cap)

    def view(self):
        n, N = self.n, self.N
        return dict(t=self.t[:n].copy(), dt=self.dt[:n].copy(), err=self.err[:n].copy(),
                    accepted=self.accepted[:n].astype(bool),
                    a=unpack_a(self.a[:n * 2 * N]).reshape(n, N),
                    mm=unpack_a(self.mm[:n * 2 * N]).reshape(n, N))


class Integrator:
    """Adaptive / replay Dormand-Prince driver around one oracle state."""

    def __init__(self, op: OracleProblem, m=None, a=None, t0: float = 0.0,
                 dt0: Optional[float] = None):
        self.op = op
        self.h = lib().orc_state_new(op.ref)
        if not self.h:
            raise MemoryError("orc_state_new")
        self.set_state(op.m0() if m is None else m, op.a0() if a is None else a, t0,
                       op.p.dt0 if dt0 is None else dt0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_state_free(h)
            self.h = None

    def set_state(self, m, a, t=0.0, dt=None):
        m = np.ascontiguousarray(m, np.float64).reshape(-1)
        a = np.ascontiguousarray(a, np.float64).reshape(-1)
        if a.size == 0:
            a = np.zeros(1)
        lib().orc_state_set(self.h, _dptr(m), _dptr(a), float(t),
                            float(self.op.p.dt0 if dt is None else dt))

    def state(self):
        m = np.empty(self.op.p.nsub * 3 * self.op.nbox)
        a = np.empty(max(2 * self.op.N, 1))
        t = C.c_double()
        dt = C.c_double()
        cnt = (C.c_long * 2)()
        lib().orc_state_get(self.h, _dptr(m), _dptr(a), C.byref(t), C.byref(dt), cnt)
        return dict(m=m, a=unpack_a(a[:2 * self.op.N]), t=t.value, dt=dt.value,
                    attempts=cnt[0], accepted=cnt[1])

    def run(self, T: float, max_attempts: int = 10 ** 9, log_cap: int = 0):
        log = Log(log_cap, self.op.N)
        rc = lib().orc_run(self.op.ref, self.h, C.byref(self.op.solver), float(T),
                           int(max_attempts), C.byref(log.s))
        return rc, log

    def run_split(self, T: float, ds: float, max_attempts: int = 10 ** 9, log_cap: int = 0):
        """Operator-split scheme (cavity RK4 with frozen overlaps, then the magnet alone) with
        interval ds, to T."""
        log = Log(log_cap, self.op.N)
        rc = lib().orc_run_split(self.op.ref, self.h, C.byref(self.op.solver), float(T),
                                 float(ds), int(max_attempts), C.byref(log.s))
        return rc, log

    def replay(self, dts, log: bool = True):
        dts = np.ascontiguousarray(dts, np.float64)
        lg = Log(len(dts) if log else 0, self.op.N)
        rc = lib().orc_replay(self.op.ref, self.h, C.byref(self.op.solver), _dptr(dts),
                              len(dts), C.byref(lg.s))
        return rc, lg


def jacobian(op: OracleProblem, m: np.ndarray, a: np.ndarray, h: float = 1e-5,
             cells: Optional[np.ndarray] = None):
    """Central-difference Jacobian of f = (dm/dt, da/dt) with respect to (m, Re a, Im a).

    Only the components of masked cells are kept (others are identically zero).  Returns
    (J, index) where index lists the flat m positions kept, followed by the 2N cavity reals.
    """
    p = op.p
    m = np.asarray(m, np.float64).reshape(-1).copy()
    a = np.asarray(a, np.float64).reshape(-1).copy()
    nbox = op.nbox
    if cells is None:
        cells = np.flatnonzero(op.mask)
    idx = np.concatenate([np.asarray(cells) + k * nbox for k in range(3 * p.nsub)])
    nv = len(idx) + 2 * op.N
    J = np.zeros((nv, nv))

    def f(mv, av):
        dm, da, _ = rhs(op, mv, av)
        return np.concatenate([dm[idx], da])

    for col in range(nv):
        if col < len(idx):
            i = idx[col]
            mp, mn = m.copy(), m.copy()
            mp[i] += h
            mn[i] -= h
            J[:, col] = (f(mp, a) - f(mn, a)) / (2 * h)
        else:
            q = col - len(idx)
            ap, an = a.copy(), a.copy()
            ap[q] += h
            an[q] -= h
            J[:, col] = (f(m, ap) - f(m, an)) / (2 * h)
    return J, idx


class Grads:
    """Parameter gradients filled by the adjoint routines (FP64): dL/d Re g~_n, dL/d Im g~_n,
    dL/d kappa_n, dL/d omega_n (each N), dL/d alpha and, with profiles, dL/d u_n(r) (N x nbox)."""

    def __init__(self, op: OracleProblem):
        N = max(op.N, 1)
        self.g_re, self.g_im = np.zeros(N), np.zeros(N)
        self.kappa, self.omega = np.zeros(N), np.zeros(N)
        self.alpha = np.zeros(1)
        self.u = np.zeros((N, op.nbox)) if op.u is not None else None
        s = _Grads()
        s.g_re, s.g_im = _dptr(self.g_re), _dptr(self.g_im)
        s.kappa, s.omega = _dptr(self.kappa), _dptr(self.omega)
        s.alpha = _dptr(self.alpha)
        s.u = _dptr(self.u) if self.u is not None else C.POINTER(C.c_double)()
        self.gb_re, self.gb_im, self.kerr = np.zeros(N), np.zeros(N), np.zeros(N)
        s.gb_re, s.gb_im = _dptr(self.gb_re), _dptr(self.gb_im)
        s.kerr = _dptr(self.kerr)
        self.pump_re, self.pump_im = np.zeros(N), np.zeros(N)
        s.pump_re, s.pump_im = _dptr(self.pump_re), _dptr(self.pump_im)
        self.s = s
        self.N = op.N

    def as_dict(self):
        N = self.N
        d = dict(g_re=self.g_re[:N].copy(), g_im=self.g_im[:N].copy(),
                 kappa=self.kappa[:N].copy(), omega=self.omega[:N].copy(),
                 alpha=float(self.alpha[0]))
        d["u"] = None if self.u is None else self.u[:N].copy()
        d["gb_re"], d["gb_im"] = self.gb_re[:N].copy(), self.gb_im[:N].copy()
        d["kerr"] = self.kerr[:N].copy()
        d["pump_re"], d["pump_im"] = self.pump_re[:N].copy(), self.pump_im[:N].copy()
        return d


def rhs_vjp(op: OracleProblem, m, a, wm, wa):
    """(df/dm)^T w, (df/da)^T w and the parameter parts at (m, a) for weights (wm, wa)."""
    m = np.ascontiguousarray(m, np.float64).reshape(-1)
    a = np.ascontiguousarray(a, np.float64).reshape(-1)
    wm = np.ascontiguousarray(wm, np.float64).reshape(-1)
    wa = np.ascontiguousarray(wa, np.float64).reshape(-1)
    if a.size == 0:
        a, wa = np.zeros(2), np.zeros(2)
    gm = np.zeros_like(m)
    ga = np.zeros(max(2 * op.N, 2))
    g = Grads(op)
    rc = lib().orc_rhs_vjp(op.ref, _dptr(m), _dptr(a), _dptr(wm), _dptr(wa), _dptr(gm),
                           _dptr(ga), C.byref(g.s))
    if rc:
        raise RuntimeError(f"orc_rhs_vjp failed: {rc}")
    d = g.as_dict()
    d["m"], d["a"] = gm, ga[:2 * op.N]
    return d


def adjoint(op: OracleProblem, m0, a0, dts, dL_da=None, dL_dm=None, t0: float = 0.0):
    """Gradient of L(a_0..a_n, m_n) through the replayed steps dts (n = len(dts)).

    dL_da: (n+1, 2N) packed reals (row i = dL/d a_i) or None; dL_dm: flat like m or None.
    Returns dict with m0, a0 (packed) and the parameter gradients of Grads.as_dict().
    """
    m0 = np.ascontiguousarray(m0, np.float64).reshape(-1)
    a0 = np.ascontiguousarray(a0, np.float64).reshape(-1)
    if a0.size == 0:
        a0 = np.zeros(2)
    dts = np.ascontiguousarray(dts, np.float64).reshape(-1)
    n = len(dts)
    null = C.POINTER(C.c_double)()
    la = None if dL_da is None else np.ascontiguousarray(dL_da, np.float64).reshape(-1)
    if la is not None and la.size != (n + 1) * 2 * op.N:
        raise ValueError("dL_da must hold (n+1) x 2N values")
    lm = None if dL_dm is None else np.ascontiguousarray(dL_dm, np.float64).reshape(-1)
    gm0 = np.zeros_like(m0)
    ga0 = np.zeros(max(2 * op.N, 2))
    g = Grads(op)
    rc = lib().orc_adjoint(op.ref, C.byref(op.solver), _dptr(m0), _dptr(a0), _dptr(dts), n,
                           _dptr(la) if la is not None else null,
                           _dptr(lm) if lm is not None else null, _dptr(gm0), _dptr(ga0),
                           C.byref(g.s), float(t0))
    if rc:
        raise RuntimeError(f"orc_adjoint failed: {rc}")
    d = g.as_dict()
    d["m0"], d["a0"] = gm0, ga0[:2 * op.N]
    return d
