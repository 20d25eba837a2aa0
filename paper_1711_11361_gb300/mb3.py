"""Python binding of the three-dimensional C ABI (include/mb3.h): argument
marshalling only; every step of the sweep runs in libmbcut.so's kernels.
Fails loudly (through ``mb``) when the library is missing."""
from __future__ import annotations

import ctypes

import numpy as np

from . import mb
from .mb import MBError, MB_OK

EXPORTS = ["mb3_create", "mb3_destroy", "mb3_last_error", "mb3_write_state", "mb3_read_state", "mb3_sweep",
           "mb3_step", "mb3_cfl_dt", "mb3_last_sweep", "mb3_flux_time", "mb3_set_precision"]


class Grid3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 6)]


class Body3(ctypes.Structure):
    _fields_ = [("nplane", ctypes.c_int), ("normals", ctypes.POINTER(ctypes.c_double)),
                ("offsets", ctypes.POINTER(ctypes.c_double)), ("bbox", ctypes.c_double * 6),
                ("U", ctypes.c_double * 3)]


lib = mb.lib
_P, _D, _I = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
for _name, (_args, _res) in {
    "mb3_create": ([ctypes.POINTER(Grid3), ctypes.c_double, ctypes.c_double, ctypes.POINTER(Body3), _I,
                    ctypes.POINTER(_P)], _I),
    "mb3_destroy": ([_P], None),
    "mb3_last_error": ([_P], ctypes.c_char_p),
    "mb3_write_state": ([_P, _D, ctypes.c_double, _D], _I),
    "mb3_read_state": ([_P, _D, _D, _D], _I),
    "mb3_sweep": ([_P, _I, ctypes.c_double], _I),
    "mb3_step": ([_P, ctypes.c_double, _D], _I),
    "mb3_cfl_dt": ([_P, _D], _I),
    "mb3_last_sweep": ([_P, _D, ctypes.POINTER(_I)], _I),
    "mb3_flux_time": ([_P, _D], _I),
    "mb3_set_precision": ([_P, _I], _I),
}.items():
    _f = getattr(lib, _name)
    _f.argtypes, _f.restype = _args, _res


def _dp(a):
    return a.ctypes.data_as(_D)


class Sim3:
    """One three-dimensional simulation from a
    :class:`paper_1711_11361_gb300.inputs.Problem3`; ``precision`` the flow
    arithmetic's (mb.FP64, the default, or mb.FP32: see set_precision)."""

    def __init__(self, prob, write_initial=True, precision=mb.FP64):
        g = Grid3()
        g.nx, g.ny, g.nz = prob.nx, prob.ny, prob.nz
        for a in range(3):
            g.lo[a], g.hi[a] = prob.lo[a], prob.hi[a]
        for q in range(6):
            g.bc[q] = prob.bc[q]
        npl = 0 if prob.normals is None else len(prob.normals)
        self._n = np.ascontiguousarray(np.zeros((1, 3)) if npl == 0 else prob.normals, dtype=np.float64)
        self._c = np.ascontiguousarray(np.zeros(1) if npl == 0 else prob.offsets, dtype=np.float64)
        b = Body3()
        b.nplane = npl
        b.normals, b.offsets = _dp(self._n), _dp(self._c)
        for q in range(6):
            b.bbox[q] = prob.bbox[q]
        for a in range(3):
            b.U[a] = prob.U[a]
        h = _P()
        r = lib.mb3_create(ctypes.byref(g), prob.gamma, prob.cfl, ctypes.byref(b), prob.uncover_mode, ctypes.byref(h))
        if r != MB_OK:
            raise MBError(r, "mb3_create failed")
        self._h = h
        self.prob = prob
        self.shape = (5, prob.nz, prob.ny, prob.nx)
        if precision != mb.FP64:
            self.set_precision(precision)
        if write_initial and prob.Q0 is not None:
            self.write_state(prob.Q0)

    def close(self):
        if getattr(self, "_h", None):
            lib.mb3_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, r):
        if r != MB_OK:
            raise MBError(r, lib.mb3_last_error(self._h).decode())
        return r

    def write_state(self, Q, t=0.0, T=(0.0, 0.0, 0.0)):
        Qc = np.ascontiguousarray(Q, dtype=np.float64).reshape(self.shape)
        Tc = np.ascontiguousarray(T, dtype=np.float64)
        self._check(lib.mb3_write_state(self._h, _dp(Qc), t, _dp(Tc)))

    def read_state(self, alpha=False, check=True):
        Q = np.empty(self.shape)
        a = np.empty(self.shape[1:]) if alpha else None
        clk = np.empty(5)
        r = lib.mb3_read_state(self._h, _dp(Q), _dp(a) if alpha else None, _dp(clk))
        if check:
            self._check(r)
        return dict(Q=Q, alpha=a, t=clk[0], T=tuple(clk[1:4]), step=int(clk[4]), status=r)

    def contents(self):
        s = self.read_state(alpha=True)
        return np.nan_to_num(s["Q"]) * s["alpha"][None]

    def sweep(self, d, dt):
        return self._check(lib.mb3_sweep(self._h, d, dt))

    def step(self, dt=0.0):
        used = ctypes.c_double()
        self._check(lib.mb3_step(self._h, dt, ctypes.byref(used)))
        return used.value

    def cfl_dt(self):
        dt = ctypes.c_double()
        self._check(lib.mb3_cfl_dt(self._h, ctypes.byref(dt)))
        return dt.value

    def set_precision(self, precision):
        """MB_FP64 (0, default) or MB_FP32 (1) flow arithmetic (mb3_set_precision)."""
        self._check(lib.mb3_set_precision(self._h, int(precision)))

    def flux_time_ms(self):
        """Device time of the last sweep's face-flux kernel (CUDA events)."""
        ms = ctypes.c_double()
        self._check(lib.mb3_flux_time(self._h, ctypes.byref(ms)))
        return ms.value

    def last_sweep(self):
        w = np.zeros(5)
        m = ctypes.c_int()
        lib.mb3_last_sweep(self._h, _dp(w), ctypes.byref(m))
        return w, m.value
