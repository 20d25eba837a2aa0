"""Plain FP64 CPU oracle for the moving-boundary cut-cell sweep (arXiv 1711.11361).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1711_11361_gb300``; both read their inputs
from ``paper_1711_11361_gb300.inputs`` (seeded problem descriptions that hold
none of the method's arithmetic).

The arithmetic lives in ``mbref.c`` (C99, compiled with -O2 -ffp-contract=off);
this module only builds it and marshals arrays through ctypes.

Functions with no independent pin are listed here (none at present): every
function below is exercised against closed forms, invariants or brute force
in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbref.c")
_LIB = os.path.join(_HERE, "libmbref.so")
_lock = threading.Lock()

EULER, ADVECTION = 0, 1
TRANSMISSIVE, REFLECTIVE, PERIODIC = 0, 1, 2
UNCOVER_DONOR, UNCOVER_FLUX_GCL = 0, 1


def build(force: bool = False) -> str:
    """Compile mbref.c into a shared library next to it (plain gcc, no FMA)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("x1", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("equation", ctypes.c_int),
        ("adv", ctypes.c_double * 2),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("uncover_mode", ctypes.c_int),
        ("npoly", ctypes.c_int),
        ("poly_start", ctypes.POINTER(ctypes.c_int)),
        ("poly_moving", ctypes.POINTER(ctypes.c_int)),
        ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double)),
        ("U", ctypes.c_double * 2), ("pivot", ctypes.c_double * 2),
        ("a0", ctypes.c_double), ("a1", ctypes.c_double), ("omega", ctypes.c_double),
        ("axisym", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        B = ctypes.POINTER(ctypes.c_ubyte)
        lib.or_create.restype = P
        lib.or_create.argtypes = [ctypes.POINTER(_Config)]
        lib.or_destroy.argtypes = [P]
        lib.or_set_state.argtypes = [P, D, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_long]
        lib.or_get_state.argtypes = [P, D, D, D]
        lib.or_sweep.argtypes = [P, ctypes.c_int, ctypes.c_double]
        lib.or_step.argtypes = [P, ctypes.c_double, D]
        lib.or_cfl_dt.argtypes = [P]
        lib.or_cfl_dt.restype = ctypes.c_double
        lib.or_geometry.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, D, B, D, D]
        lib.or_swept.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, D]
        lib.or_hllc.argtypes = [ctypes.c_double, ctypes.c_int, D, D, D]
        lib.or_wall_state.argtypes = [ctypes.c_double, D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, D, D, D, D]
        lib.or_status.argtypes = [P]
        lib.or_last_sweep.argtypes = [P, D]
        lib.or_stab_face.argtypes = [ctypes.c_int, ctypes.c_double, D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     D, ctypes.c_int, ctypes.c_double, ctypes.c_double, D, D]
        lib.or_cover_uncover.argtypes = [ctypes.c_int] * 7 + [D, D, D, D, B]
        lib.or_safeguard.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, D, D, B, D]
        lib.or_last_faces.argtypes = [P, D]
        lib.or_last_wall.argtypes = [P, D]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def hllc(gamma: float, d: int, qL, qR) -> np.ndarray:
    """HLLC flux along direction d between conserved states qL and qR."""
    lib = _load()
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    F = np.zeros(4)
    lib.or_hllc(gamma, d, _dp(qL), _dp(qR), _dp(F))
    return F


def wall_state(gamma: float, q, n, w):
    """(rho*, p*, u*x, u*y) of the moving-wall Riemann problem for cell state q."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = [ctypes.c_double() for _ in range(4)]
    lib.or_wall_state(gamma, _dp(q), float(n[0]), float(n[1]), float(w[0]), float(w[1]),
                      *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def stab_face(bf, F, left=None, right=None):
    """Stabilised flux (times the face aperture bf) of one face with standard
    flux F.  left / right: None, or (bfar, d, FB) of a neighbour with wall
    data: the aperture of its far face, its shielded distance and its
    boundary flux."""
    lib = _load()
    F = np.ascontiguousarray(F, dtype=np.float64)
    nc = F.size
    z = np.zeros(nc)
    bl, dl, fbl = left if left is not None else (0.0, 0.0, z)
    br, dr, fbr = right if right is not None else (0.0, 0.0, z)
    fbl = np.ascontiguousarray(fbl, dtype=np.float64)
    fbr = np.ascontiguousarray(fbr, dtype=np.float64)
    out = np.zeros(nc)
    lib.or_stab_face(nc, bf, _dp(F), 1 if left is not None else 0, bl, dl, _dp(fbl),
                     1 if right is not None else 0, br, dr, _dp(fbr), _dp(out))
    return out


def cover_uncover(alphaA, alphaB, C, mode=UNCOVER_DONOR, periodic=(False, False), open_sides=0):
    """Covering / uncovering redistribution of the contents C (nc, ny, nx)
    between the poses with volume fractions alphaA and alphaB (ny, nx)
    (open_sides: bit mask of transmissive sides x-low, x-high, y-low,
    y-high); returns (new contents, status, updated flags)."""
    lib = _load()
    aA = np.ascontiguousarray(alphaA, dtype=np.float64)
    aB = np.ascontiguousarray(alphaB, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    if C.ndim == 2:
        C = C[None]
    nc, ny, nx = C.shape
    Cn = np.empty_like(C)
    upd = np.zeros((ny, nx), dtype=np.uint8)
    r = lib.or_cover_uncover(nx, ny, int(periodic[0]), int(periodic[1]), int(open_sides), nc, mode, _dp(aA),
                             _dp(aB), _dp(C),
                             _dp(Cn), upd.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return Cn, r, upd


def safeguard(alphaB, C, updated=None, gamma=1.4, periodic=(False, False), alphaA=None):
    """Positivity safeguard on Euler contents C (4, ny, nx); returns (merged
    contents, cells merged).  With alphaA (the volume fractions at the start
    of the sweep), cells that kept less than 1% of their volume also seed the
    first merge."""
    lib = _load()
    aB = np.ascontiguousarray(alphaB, dtype=np.float64)
    aA = None if alphaA is None else np.ascontiguousarray(alphaA, dtype=np.float64)
    Cn = np.array(C, dtype=np.float64, order="C", copy=True)
    _, ny, nx = Cn.shape
    upd = np.ascontiguousarray(np.ones((ny, nx), dtype=np.uint8) if updated is None else updated, dtype=np.uint8)
    m = lib.or_safeguard(nx, ny, int(periodic[0]), int(periodic[1]), gamma, None if aA is None else _dp(aA), _dp(aB),
                         upd.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _dp(Cn))
    return Cn, m


class Oracle:
    """One oracle simulation built from a :class:`paper_1711_11361_gb300.inputs.Problem`."""

    def __init__(self, prob):
        self._lib = _load()
        self.prob = prob
        self.nx, self.ny = prob.nx, prob.ny
        self.nc = 4 if prob.equation == EULER else 1
        starts = [0]
        for poly in prob.polygons:
            starts.append(starts[-1] + len(poly))
        self._pstart = np.array(starts, dtype=np.int32)
        self._pmov = np.array(prob.moving if prob.polygons else [0], dtype=np.int32)
        if prob.polygons:
            allv = np.concatenate([np.asarray(p, dtype=np.float64) for p in prob.polygons])
        else:
            allv = np.zeros((1, 2))
        self._vx = np.ascontiguousarray(allv[:, 0])
        self._vy = np.ascontiguousarray(allv[:, 1])
        c = _Config()
        c.nx, c.ny = prob.nx, prob.ny
        c.x0, c.y0, c.x1, c.y1 = prob.x0, prob.y0, prob.x1, prob.y1
        for k in range(4):
            c.bc[k] = prob.bc[k]
        c.equation = prob.equation
        c.adv[0], c.adv[1] = prob.adv
        c.gamma, c.cfl = prob.gamma, prob.cfl
        c.uncover_mode = prob.uncover_mode
        c.npoly = len(prob.polygons)
        c.poly_start = self._pstart.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        c.poly_moving = self._pmov.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        c.vx, c.vy = _dp(self._vx), _dp(self._vy)
        c.U[0], c.U[1] = prob.U
        c.pivot[0], c.pivot[1] = prob.pivot
        c.a0, c.a1, c.omega = prob.a0, prob.a1, prob.omega
        c.axisym = 1 if getattr(prob, "axisym", False) else 0
        self._cfg = c
        self._h = self._lib.or_create(ctypes.byref(c))
        if not self._h:
            raise ValueError("oracle rejected the problem")
        if prob.Q0 is not None:
            self.set_state(prob.Q0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    # state -----------------------------------------------------------------
    def set_state(self, Q, t=0.0, X=0.0, Y=0.0, step=0):
        Q = np.ascontiguousarray(Q, dtype=np.float64).reshape(self.nc, self.ny, self.nx)
        self._lib.or_set_state(self._h, _dp(Q), t, X, Y, step)

    def state(self):
        Q = np.empty((self.nc, self.ny, self.nx))
        self._lib.or_get_state(self._h, _dp(Q), None, None)
        return Q

    def alpha(self):
        a = np.empty((self.ny, self.nx))
        self._lib.or_get_state(self._h, None, _dp(a), None)
        return a

    def clock(self):
        o = np.empty(4)
        self._lib.or_get_state(self._h, None, None, _dp(o))
        return dict(t=o[0], X=o[1], Y=o[2], step=int(o[3]))

    @property
    def status(self):
        return self._lib.or_status(self._h)

    # stepping --------------------------------------------------------------
    def sweep(self, d: int, dt: float) -> int:
        return self._lib.or_sweep(self._h, d, dt)

    def step(self, dt: float = 0.0):
        out = ctypes.c_double()
        r = self._lib.or_step(self._h, dt, ctypes.byref(out))
        return r, out.value

    def last_sweep(self):
        """(sum of the last sweep's wall terms per component, cells merged)."""
        w = np.zeros(4)
        m = self._lib.or_last_sweep(self._h, _dp(w))
        return w[: self.nc], m

    def last_faces(self):
        """(direction, time-averaged apertures of the last sweep's faces)."""
        nx, ny = self.nx, self.ny
        buf = np.zeros(max((nx + 1) * ny, nx * (ny + 1)))
        d = self._lib.or_last_faces(self._h, _dp(buf))
        if d < 0:
            return d, None
        return d, (buf[: (nx + 1) * ny].reshape(ny, nx + 1) if d == 0 else buf[: nx * (ny + 1)].reshape(ny + 1, nx))

    def last_wall(self):
        """Wall data of the last sweep per cell: dict of (ny, nx) arrays has,
        d, nx, ny (normal), wx, wy (wall velocity at the mid pose)."""
        out = np.zeros((self.ny, self.nx, 6))
        self._lib.or_last_wall(self._h, _dp(out))
        return {k: out[..., i] for i, k in enumerate(("has", "d", "n_x", "n_y", "wx", "wy"))}

    def cfl_dt(self) -> float:
        return self._lib.or_cfl_dt(self._h)

    # geometry --------------------------------------------------------------
    def geometry(self, X=0.0, Y=0.0, theta=0.0):
        nx, ny = self.nx, self.ny
        a = np.empty((ny, nx))
        t = np.empty((ny, nx), dtype=np.uint8)
        bx = np.empty((ny, nx + 1))
        by = np.empty((ny + 1, nx))
        self._lib.or_geometry(self._h, X, Y, theta, _dp(a),
                              t.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _dp(bx), _dp(by))
        return a, t, bx, by

    def swept(self, d, delta, X=0.0, Y=0.0, theta=0.0):
        nx, ny = self.nx, self.ny
        out = np.empty((ny, nx + 1)) if d == 0 else np.empty((ny + 1, nx))
        self._lib.or_swept(self._h, d, X, Y, theta, delta, _dp(out))
        return out

    # diagnostics -------------------------------------------------------------
    def contents(self):
        """alpha * Q with solid cells set to 0 (per component)."""
        a = self.alpha()
        Q = self.state()
        return np.where(a[None] > 0, a[None] * np.nan_to_num(Q), 0.0)
