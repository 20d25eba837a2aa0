"""Three-dimensional FP64 CPU oracle (``mb3ref.c``): the dimensionally split
moving-boundary method with x, y and z sweeps (Sec. II.C.4, eqs.
Klein2DcompleteMovingMethod2a-c) for one convex polyhedral body translating
at constant velocity.  TEST INFRASTRUCTURE ONLY, under the same rules as
``oracle``: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may use it; it shares no code with the CUDA library.

Pins: ``tests/test_oracle_3d.py`` (closed-form volumes, apertures and swept
apertures, the body's volume, uniform flow, conservation, and the reduction
to the pinned two-dimensional oracle for z- and x-invariant prisms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mb3ref.c")
_LIB = os.path.join(_HERE, "libmb3ref.so")
_lock = threading.Lock()
MAXP = 32


def build(force: bool = False) -> str:
    """Compile mb3ref.c into a shared library next to it (plain gcc, no FMA)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
        ("x1", ctypes.c_double), ("y1", ctypes.c_double), ("z1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("nplane", ctypes.c_int),
        ("pn", ctypes.c_double * (3 * MAXP)),
        ("pc", ctypes.c_double * MAXP),
        ("U", ctypes.c_double * 3),
        ("uncover_mode", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        B = ctypes.POINTER(ctypes.c_ubyte)
        lib.o3_create.restype = P
        lib.o3_create.argtypes = [ctypes.POINTER(_Config), D]
        lib.o3_destroy.argtypes = [P]
        lib.o3_set_state.argtypes = [P, D, ctypes.c_double, D, ctypes.c_long]
        lib.o3_get_state.argtypes = [P, D, D, D]
        lib.o3_sweep.argtypes = [P, ctypes.c_int, ctypes.c_double]
        lib.o3_step.argtypes = [P, ctypes.c_double]
        lib.o3_cfl_dt.argtypes = [P]
        lib.o3_cfl_dt.restype = ctypes.c_double
        lib.o3_geometry.argtypes = [P, D, D, B, D, D, D]
        lib.o3_swept.argtypes = [P, ctypes.c_int, D, ctypes.c_double, D]
        lib.o3_last_sweep.argtypes = [P, D]
        lib.o3_last_wall.argtypes = [P, D]
        lib.o3_solid_volume.argtypes = [P, D, D, D]
        lib.o3_solid_volume.restype = ctypes.c_double
        lib.o3_cover_uncover.argtypes = [P, D, D, D, D, B]
        lib.o3_safeguard.argtypes = [P, D, D, B, D]
        lib.o3_hllc.argtypes = [ctypes.c_double, ctypes.c_int, D, D, D]
        lib.o3_wall_state.argtypes = [ctypes.c_double, D, D, D, D, D, D]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(v):
    return np.ascontiguousarray(v, dtype=np.float64)


def hllc(gamma, d, qL, qR):
    F = np.zeros(5)
    _load().o3_hllc(gamma, d, _dp(_vec(qL)), _dp(_vec(qR)), _dp(F))
    return F


def wall_state(gamma, q, n, w):
    rs, ps, us = ctypes.c_double(), ctypes.c_double(), np.zeros(3)
    _load().o3_wall_state(gamma, _dp(_vec(q)), _dp(_vec(n)), _dp(_vec(w)), ctypes.byref(rs), ctypes.byref(ps),
                          _dp(us))
    return rs.value, ps.value, us


class Oracle3:
    """One three-dimensional oracle simulation built from a
    :class:`paper_1711_11361_gb300.inputs.Problem3`."""

    def __init__(self, prob):
        lib = _load()
        c = _Config()
        c.nx, c.ny, c.nz = prob.nx, prob.ny, prob.nz
        c.x0, c.y0, c.z0 = prob.lo
        c.x1, c.y1, c.z1 = prob.hi
        c.gamma, c.cfl = prob.gamma, prob.cfl
        for k in range(6):
            c.bc[k] = prob.bc[k]
        npl = 0 if prob.normals is None else len(prob.normals)
        if npl > MAXP:
            raise ValueError(f"at most {MAXP} planes")
        c.nplane = npl
        for f in range(npl):
            for a in range(3):
                c.pn[3 * f + a] = float(prob.normals[f][a])
            c.pc[f] = float(prob.offsets[f])
        for a in range(3):
            c.U[a] = prob.U[a]
        c.uncover_mode = prob.uncover_mode
        self._cfg = c
        self._bb = _vec(prob.bbox)
        self._h = lib.o3_create(ctypes.byref(c), _dp(self._bb))
        if not self._h:
            raise ValueError("o3_create rejected the configuration")
        self.nx, self.ny, self.nz = prob.nx, prob.ny, prob.nz
        self.n = prob.nx * prob.ny * prob.nz
        if prob.Q0 is not None:
            self.set_state(prob.Q0)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.o3_destroy(self._h)
            self._h = None

    def set_state(self, Q, t=0.0, T=(0.0, 0.0, 0.0), step=0):
        Qc = np.ascontiguousarray(Q, dtype=np.float64).reshape(5, self.nz, self.ny, self.nx)
        _lib.o3_set_state(self._h, _dp(Qc), t, _dp(_vec(T)), step)

    def state(self):
        Q = np.empty((5, self.nz, self.ny, self.nx))
        _lib.o3_get_state(self._h, _dp(Q), None, None)
        return Q

    def alpha(self):
        a = np.empty((self.nz, self.ny, self.nx))
        _lib.o3_get_state(self._h, None, _dp(a), None)
        return a

    def contents(self):
        a = self.alpha()
        return np.nan_to_num(self.state()) * a[None]

    def clock(self):
        c = np.empty(5)
        _lib.o3_get_state(self._h, None, None, _dp(c))
        return dict(t=c[0], T=tuple(c[1:4]), step=int(c[4]))

    def sweep(self, d, dt):
        return _lib.o3_sweep(self._h, d, dt)

    def step(self, dt=0.0):
        if dt <= 0.0:
            dt = self.cfl_dt()
        return _lib.o3_step(self._h, dt), dt

    def cfl_dt(self):
        return _lib.o3_cfl_dt(self._h)

    def last_sweep(self):
        w = np.zeros(5)
        m = _lib.o3_last_sweep(self._h, _dp(w))
        return w, m

    def last_wall(self):
        """Wall data of the last sweep per cell: dict of (nz, ny, nx) arrays
        has, d, n_x, n_y, n_z."""
        out = np.zeros((self.nz, self.ny, self.nx, 5))
        _lib.o3_last_wall(self._h, _dp(out))
        return {k: out[..., i] for i, k in enumerate(("has", "d", "n_x", "n_y", "n_z"))}

    def geometry(self, T=(0.0, 0.0, 0.0)):
        nx, ny, nz = self.nx, self.ny, self.nz
        a = np.empty((nz, ny, nx))
        t = np.empty((nz, ny, nx), dtype=np.uint8)
        bx = np.empty((nz, ny, nx + 1))
        by = np.empty((nz, ny + 1, nx))
        bz = np.empty((nz + 1, ny, nx))
        _lib.o3_geometry(self._h, _dp(_vec(T)), _dp(a), t.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                         _dp(bx), _dp(by), _dp(bz))
        return a, t, (bx, by, bz)

    def swept(self, d, delta, T=(0.0, 0.0, 0.0)):
        nx, ny, nz = self.nx, self.ny, self.nz
        shape = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][d]
        out = np.empty(shape)
        _lib.o3_swept(self._h, d, _dp(_vec(T)), delta, _dp(out))
        return out

    def cover_uncover(self, alphaA, alphaB, C):
        """The covering / uncovering step alone (Sec. II.C.5) on given fields
        of shape (nz, ny, nx) and contents (5, nz, ny, nx): (status, Cn,
        updated flags)."""
        aA, aB = _vec(alphaA).reshape(-1), _vec(alphaB).reshape(-1)
        Cc = _vec(C).reshape(-1)
        Cn = np.empty_like(Cc)
        upd = np.zeros(self.n, dtype=np.uint8)
        r = _lib.o3_cover_uncover(self._h, _dp(aA), _dp(aB), _dp(Cc), _dp(Cn),
                                  upd.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return r, Cn.reshape(5, self.nz, self.ny, self.nx), upd.reshape(self.nz, self.ny, self.nx)

    def safeguard(self, alphaA, alphaB, updated, Cn):
        """The positivity safeguard alone on given fields: (cells merged, Cn)."""
        aA, aB = _vec(alphaA).reshape(-1), _vec(alphaB).reshape(-1)
        up = np.ascontiguousarray(updated, dtype=np.uint8).reshape(-1)
        C = _vec(Cn).reshape(-1).copy()
        m = _lib.o3_safeguard(self._h, _dp(aA), _dp(aB), up.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _dp(C))
        return m, C.reshape(5, self.nz, self.ny, self.nx)

    def solid_volume(self, lo, hi, T=(0.0, 0.0, 0.0)):
        return _lib.o3_solid_volume(self._h, _dp(_vec(T)), _dp(_vec(lo)), _dp(_vec(hi)))
