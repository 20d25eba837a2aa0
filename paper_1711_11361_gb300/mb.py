"""ctypes binding of libmbcut.so (C ABI in include/mb.h).

Argument marshalling only: every step of the sweep runs in the CUDA library.
Importing this module loads the library and raises ImportError if it has not
been built (``python -c "import __graft_entry__ as g; g.build()"``); there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmbcut.so")

MB_OK, MB_E_INVAL, MB_E_NOMEM, MB_E_CUDA, MB_E_UNSTABLE, MB_E_TIMEOUT, MB_E_STATE, MB_E_CAPACITY = 0, -1, -2, -3, -4, -5, -6, -7
FP64, FP32 = 0, 1

EXPORTS = ["mb_create", "mb_batch_create", "mb_destroy", "mb_last_error", "mb_set_stream", "mb_write_state",
           "mb_read_state", "mb_step", "mb_sweep", "mb_run", "mb_sync", "mb_info", "mb_diagnostics",
           "mb_enable_timing", "mb_kernel_time", "mb_band_records", "mb_band_record_size",
           "mb_cut_cells_noalloc", "mb_noalloc_last_error", "mb_batch_add", "mb_batch_remove", "mb_instance_bytes",
           "mb_request_bytes", "mb_server_create", "mb_server_destroy", "mb_server_last_error", "mb_server_submit",
           "mb_server_tick", "mb_server_query", "mb_server_request_error", "mb_autotune", "mb_set_overlap",
           "mb_write_states", "mb_read_states", "mb_graph_kernels", "mb_set_sweep_event",
           "mb_merge_count", "mb_fp64_rate", "mb_probe", "mb_write_states_f32", "mb_read_states_f32"]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("x1", ctypes.c_double), ("y1", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("equation", ctypes.c_int), ("adv", ctypes.c_double * 2),
                ("cfl", ctypes.c_double), ("uncover_mode", ctypes.c_int), ("precision", ctypes.c_int)]


class Body(ctypes.Structure):
    _fields_ = [("npoly", ctypes.c_int), ("poly_start", ctypes.POINTER(ctypes.c_int)),
                ("poly_moving", ctypes.POINTER(ctypes.c_int)),
                ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double))]


class Motion(ctypes.Structure):
    _fields_ = [("U", ctypes.c_double * 2), ("pivot", ctypes.c_double * 2),
                ("a0", ctypes.c_double), ("a1", ctypes.c_double), ("omega", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("grid", Grid), ("gamma", ctypes.c_double), ("body", Body), ("motion", Motion),
                ("Q0", ctypes.POINTER(ctypes.c_double)), ("t0", ctypes.c_double), ("nsteps", ctypes.c_int),
                ("Qout", ctypes.POINTER(ctypes.c_double))]


class MBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mb error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(the CUDA library is the only implementation; there is no fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "mb_create": ([ctypes.POINTER(Grid), ctypes.c_double, ctypes.POINTER(Body), ctypes.POINTER(Motion), PP], I),
        "mb_batch_create": ([I, ctypes.POINTER(Grid), D, ctypes.POINTER(Body), ctypes.POINTER(Motion), PP], I),
        "mb_destroy": ([P], None),
        "mb_last_error": ([P], ctypes.c_char_p),
        "mb_set_stream": ([P, P], I),
        "mb_write_state": ([P, I, D, ctypes.c_double], I),
        "mb_read_state": ([P, I, D, D, D], I),
        "mb_step": ([P, ctypes.c_double, D], I),
        "mb_sweep": ([P, I, ctypes.c_double], I),
        "mb_run": ([P, I, ctypes.c_double], I),
        "mb_sync": ([P], I),
        "mb_info": ([P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "mb_diagnostics": ([P, I, D], I),
        "mb_enable_timing": ([P, I], I),
        "mb_kernel_time": ([P, D, ctypes.POINTER(I)], I),
        "mb_band_records": ([P, I, P, I, ctypes.POINTER(I)], I),
        "mb_band_record_size": ([], I),
        "mb_cut_cells_noalloc": ([ctypes.POINTER(Grid), ctypes.POINTER(Body), ctypes.POINTER(Motion), ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, P, P, P], I),
        "mb_noalloc_last_error": ([], ctypes.c_char_p),
        "mb_batch_add": ([P, ctypes.POINTER(Grid), ctypes.c_double, ctypes.POINTER(Body), ctypes.POINTER(Motion),
                          ctypes.POINTER(I)], I),
        "mb_batch_remove": ([P, I], I),
        "mb_instance_bytes": ([P, I], ctypes.c_size_t),
        "mb_request_bytes": ([ctypes.POINTER(Grid), ctypes.POINTER(Body), ctypes.POINTER(Motion)], ctypes.c_size_t),
        "mb_server_create": ([I, I, ctypes.c_double, I, PP], I),
        "mb_server_destroy": ([P], None),
        "mb_server_last_error": ([P], ctypes.c_char_p),
        "mb_server_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(I)], I),
        "mb_server_tick": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "mb_server_query": ([P, I, ctypes.POINTER(I), D], I),
        "mb_server_request_error": ([P, I], ctypes.c_char_p),
        "mb_autotune": ([P, D], I),
        "mb_set_overlap": ([P, I], I),
        "mb_write_states": ([P, ctypes.POINTER(D), D], I),
        "mb_read_states": ([P, ctypes.POINTER(D), D], I),
        "mb_write_states_f32": ([P, ctypes.POINTER(ctypes.POINTER(ctypes.c_float)), D], I),
        "mb_read_states_f32": ([P, ctypes.POINTER(ctypes.POINTER(ctypes.c_float)), D], I),
        "mb_graph_kernels": ([P, ctypes.POINTER(I)], I),
        "mb_set_sweep_event": ([P, P], I),
        "mb_merge_count": ([P, I, ctypes.POINTER(ctypes.c_longlong)], I),
        "mb_fp64_rate": ([P, D], I),
        "mb_probe": ([P, I, I, ctypes.POINTER(ctypes.c_int), D], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _marshal(prob: inputs.Problem, precision: int):
    g = Grid()
    g.nx, g.ny = prob.nx, prob.ny
    g.x0, g.y0, g.x1, g.y1 = prob.x0, prob.y0, prob.x1, prob.y1
    for k in range(4):
        g.bc[k] = prob.bc[k]
    g.equation = 2 if getattr(prob, "axisym", False) else prob.equation   # MB_EULER_AXISYM
    g.adv[0], g.adv[1] = prob.adv
    g.cfl = prob.cfl
    g.uncover_mode = prob.uncover_mode
    g.precision = precision
    starts = [0]
    for poly in prob.polygons:
        starts.append(starts[-1] + len(poly))
    keep = {}
    keep["ps"] = np.array(starts, dtype=np.int32)
    keep["pm"] = np.array(prob.moving if prob.polygons else [0], dtype=np.int32)
    allv = np.concatenate([np.asarray(p, dtype=np.float64) for p in prob.polygons]) if prob.polygons else np.zeros((1, 2))
    keep["vx"] = np.ascontiguousarray(allv[:, 0])
    keep["vy"] = np.ascontiguousarray(allv[:, 1])
    b = Body()
    b.npoly = len(prob.polygons)
    b.poly_start = keep["ps"].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    b.poly_moving = keep["pm"].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    b.vx, b.vy = _dp(keep["vx"]), _dp(keep["vy"])
    m = Motion()
    m.U[0], m.U[1] = prob.U
    m.pivot[0], m.pivot[1] = prob.pivot
    m.a0, m.a1, m.omega = prob.a0, prob.a1, prob.omega
    return g, b, m, keep


class Sim:
    """A batch of instances advancing together on the GPU."""

    def __init__(self, problems, precision: int = FP64, write_initial: bool = True):
        if isinstance(problems, inputs.Problem):
            problems = [problems]
        self.problems = list(problems)
        n = len(self.problems)
        gs, bs, ms, self._keep = (Grid * n)(), (Body * n)(), (Motion * n)(), []
        gam = np.array([p.gamma for p in self.problems], dtype=np.float64)
        for k, p in enumerate(self.problems):
            g, b, m, keep = _marshal(p, precision)
            gs[k], bs[k], ms[k] = g, b, m
            self._keep.append(keep)
        h = ctypes.c_void_p()
        r = lib.mb_batch_create(n, gs, _dp(gam), bs, ms, ctypes.byref(h))
        if r != MB_OK:
            raise MBError(r, lib.mb_last_error(None).decode())
        self._h = h
        self.n = n
        self.precision = precision
        if write_initial:
            if all(p.Q0 is not None for p in self.problems):
                self.write_states([p.Q0 for p in self.problems])
            else:
                for k, p in enumerate(self.problems):
                    if p.Q0 is not None:
                        self.write_state(k, p.Q0)

    def _check(self, r):
        if r != MB_OK:
            raise MBError(r, lib.mb_last_error(self._h).decode())
        return r

    def close(self):
        if getattr(self, "_h", None):
            lib.mb_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_stream(self, stream_handle: int):
        self._check(lib.mb_set_stream(self._h, ctypes.c_void_p(stream_handle)))

    def write_state(self, inst, Q, t=0.0):
        p = self.problems[inst]
        Q = np.ascontiguousarray(Q, dtype=np.float64).reshape(p.nc, p.ny, p.nx)
        self._check(lib.mb_write_state(self._h, inst, _dp(Q), t))

    @staticmethod
    def _ptrs(arrays, ctype=ctypes.c_double):
        # numpy arrays, or addresses (ints) of host buffers such as pinned
        # torch tensors' data_ptr()
        T = ctypes.POINTER(ctype)
        return (T * len(arrays))(*[ctypes.cast(a, T) if isinstance(a, int) else a.ctypes.data_as(T)
                                   for a in arrays])

    def write_states(self, Qs, t=None, dtype=np.float64):
        """Every instance's state in one call (mb_write_states, or
        mb_write_states_f32 for dtype float32).  Qs[k]: a C-contiguous array
        of shape (nc, ny, nx), or the address of such a host buffer of that
        dtype; t: times (default 0)."""
        if len(Qs) != self.n:
            raise ValueError("one state per instance")
        f32 = np.dtype(dtype) == np.float32
        keep = []
        for k, Q in enumerate(Qs):
            if not isinstance(Q, int):
                p = self.problems[k]
                Q = np.ascontiguousarray(Q, dtype=np.float32 if f32 else np.float64).reshape(p.nc, p.ny, p.nx)
            keep.append(Q)
        tt = None if t is None else np.ascontiguousarray(t, dtype=np.float64)
        fn = lib.mb_write_states_f32 if f32 else lib.mb_write_states
        ptrs = self._ptrs(keep, ctypes.c_float if f32 else ctypes.c_double)
        self._check(fn(self._h, ptrs, _dp(tt) if tt is not None else None))

    def read_states(self, out=None, check=True, dtype=np.float64):
        """Every instance's state in one call (mb_read_states, or
        mb_read_states_f32 for dtype float32) into out (as for write_states)
        or new arrays; returns (states, clocks (n, 4), status)."""
        f32 = np.dtype(dtype) == np.float32
        if out is None:
            out = [np.empty((p.nc, p.ny, p.nx), dtype=np.float32 if f32 else np.float64) for p in self.problems]
        clk = np.empty((self.n, 4))
        fn = lib.mb_read_states_f32 if f32 else lib.mb_read_states
        r = fn(self._h, self._ptrs(out, ctypes.c_float if f32 else ctypes.c_double), _dp(clk))
        if check:
            self._check(r)
        return out, clk, r

    def read_state(self, inst=0, alpha=False, check=True):
        p = self.problems[inst]
        Q = np.empty((p.nc, p.ny, p.nx))
        a = np.empty((p.ny, p.nx)) if alpha else None
        clk = np.empty(4)
        r = lib.mb_read_state(self._h, inst, _dp(Q), _dp(a) if alpha else None, _dp(clk))
        if check:
            self._check(r)
        out = dict(Q=Q, t=clk[0], X=clk[1], Y=clk[2], step=int(clk[3]), status=r)
        if alpha:
            out["alpha"] = a
        return out

    def step(self, dt=0.0, report=False):
        if report:
            out = np.empty(self.n)
            self._check(lib.mb_step(self._h, dt, _dp(out)))
            return out
        self._check(lib.mb_step(self._h, dt, None))

    def sweep(self, d, dt):
        self._check(lib.mb_sweep(self._h, d, dt))

    def run(self, nsteps, dt=0.0):
        self._check(lib.mb_run(self._h, nsteps, dt))

    def sync(self):
        return self._check(lib.mb_sync(self._h))

    def diagnostics(self, inst=0):
        o = np.zeros(6)
        self._check(lib.mb_diagnostics(self._h, inst, _dp(o)))
        return dict(wall=o[:4], mixed=int(o[4]), band=int(o[5]))

    def probe(self, inst, cells):
        """States at the given (i, j) cells between steps (mb_probe): array (nc, len(cells))."""
        ij = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1))
        n = ij.size // 2
        out = np.empty((self.problems[inst].nc, n))
        self._check(lib.mb_probe(self._h, inst, n, ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out)))
        return out

    def merge_count(self, inst=0):
        """Cells merged by the positivity safeguard since the instance's state was written (mb_merge_count)."""
        c = ctypes.c_longlong()
        self._check(lib.mb_merge_count(self._h, inst, ctypes.byref(c)))
        return c.value

    def autotune(self):
        """Tune the bulk kernels' launch shapes (mb_autotune); returns the choice."""
        r = np.zeros(8)
        self._check(lib.mb_autotune(self._h, _dp(r)))
        return dict(x_cta=int(r[0]), y_cta=int(r[1]), y_rows=int(r[2]), x_ms=r[3], y_ms=r[4],
                    x_min_ctas=int(r[5]), y_min_ctas=int(r[6]), x_ring_chunks=int(r[7]))

    def set_overlap(self, on=True):
        """Overlap of the bulk pass with the geometry and band fluxes (mb_set_overlap)."""
        self._check(lib.mb_set_overlap(self._h, 1 if on else 0))

    def graph_kernels(self):
        """Kernel launches per step of the step graph captured last (mb_graph_kernels)."""
        k = ctypes.c_int()
        self._check(lib.mb_graph_kernels(self._h, ctypes.byref(k)))
        return k.value

    def set_sweep_event(self, event_handle: int):
        """Record a CUDA event between the two sweeps of each step (mb_set_sweep_event; 0: none)."""
        self._check(lib.mb_set_sweep_event(self._h, ctypes.c_void_p(event_handle)))

    def enable_timing(self, on=True):
        self._check(lib.mb_enable_timing(self._h, 1 if on else 0))

    def kernel_time(self):
        ms = ctypes.c_double()
        n = ctypes.c_int()
        self._check(lib.mb_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def add(self, prob: inputs.Problem, write_initial: bool = True) -> int:
        """Append an instance between steps (mb_batch_add); returns its index."""
        g, b, m, keep = _marshal(prob, self.precision)
        k = ctypes.c_int()
        self._check(lib.mb_batch_add(self._h, ctypes.byref(g), prob.gamma, ctypes.byref(b), ctypes.byref(m),
                                     ctypes.byref(k)))
        self.problems.append(prob)
        self._keep.append(keep)
        self.n += 1
        if write_initial and prob.Q0 is not None:
            self.write_state(k.value, prob.Q0)
        return k.value

    def remove(self, inst: int):
        """Remove an instance between steps (mb_batch_remove); later indices move down."""
        self._check(lib.mb_batch_remove(self._h, inst))
        del self.problems[inst]
        del self._keep[inst]
        self.n -= 1

    def band_records(self, inst=0):
        """Raw band records of the last sweep as a numpy structured array."""
        cnt = ctypes.c_int()
        self._check(lib.mb_band_records(self._h, inst, None, 0, ctypes.byref(cnt)))
        out = np.zeros(cnt.value, dtype=BAND_DTYPE)
        if cnt.value:
            self._check(lib.mb_band_records(self._h, inst, out.ctypes.data_as(ctypes.c_void_p), cnt.value,
                                            ctypes.byref(cnt)))
        return out


def cut_cells_noalloc(prob: inputs.Problem, X: float, Y: float, theta: float, alpha_ptr: int, class_ptr: int,
                      stream: int = 0):
    """Volume fractions and class bytes of `prob`'s body posed at (X, Y,
    theta) into caller-owned device arrays, without any device allocation
    by the library (see mb_cut_cells_noalloc in include/mb.h)."""
    g, b, m, keep = _marshal(prob, FP64)
    r = lib.mb_cut_cells_noalloc(ctypes.byref(g), ctypes.byref(b), ctypes.byref(m), X, Y, theta,
                                 ctypes.c_void_p(alpha_ptr), ctypes.c_void_p(class_ptr), ctypes.c_void_p(stream))
    if r != MB_OK:
        raise MBError(r, lib.mb_noalloc_last_error().decode())


def fp64_rate(stream: int = 0) -> float:
    """Measured FP64 fused multiply-adds per second of this GPU (mb_fp64_rate)."""
    r = ctypes.c_double()
    rc = lib.mb_fp64_rate(ctypes.c_void_p(stream), ctypes.byref(r))
    if rc != MB_OK:
        raise MBError(rc, "mb_fp64_rate failed")
    return r.value


class Server:
    """Continuous-batching request loop (mb_server_* in include/mb.h)."""

    QUEUED, RUNNING, DONE = 0, 1, 2

    def __init__(self, precision=FP32, equation=0, budget_bytes=32 * 2 ** 30, max_active=64):
        h = ctypes.c_void_p()
        r = lib.mb_server_create(precision, equation, float(budget_bytes), max_active, ctypes.byref(h))
        if r != MB_OK:
            raise MBError(r, "bad server arguments")
        self._h = h
        self.precision = precision
        self._keep = {}
        self.out = {}

    def close(self):
        if getattr(self, "_h", None):
            lib.mb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, r):
        if r != MB_OK:
            raise MBError(r, lib.mb_server_last_error(self._h).decode())

    def submit(self, prob: inputs.Problem, nsteps: int, Q0=None, t0=0.0, keep_result=True) -> int:
        """Queue a request (the library copies its description and initial
        state).  keep_result=False: the final state is not returned."""
        g, b, m, keep = _marshal(prob, self.precision)
        Q0 = np.ascontiguousarray(prob.Q0 if Q0 is None else Q0, dtype=np.float64)
        out = np.full((prob.nc, prob.ny, prob.nx), np.nan) if keep_result else None
        req = Request(g, prob.gamma, b, m, _dp(Q0), t0, nsteps, _dp(out) if keep_result else None)
        k = ctypes.c_int()
        self._check(lib.mb_server_submit(self._h, ctypes.byref(req), ctypes.byref(k)))
        if keep_result:
            self.out[k.value] = out
        return k.value

    def tick(self):
        a, q, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib.mb_server_tick(self._h, ctypes.byref(a), ctypes.byref(q), ctypes.byref(d)))
        return a.value, q.value, d.value

    def query(self, rid: int):
        st = ctypes.c_int()
        info = np.zeros(5)
        self._check(lib.mb_server_query(self._h, rid, ctypes.byref(st), _dp(info)))
        return dict(state=st.value, t_submit=info[0], t_admit=info[1], t_done=info[2], steps=int(info[3]),
                    bytes=int(info[4]), error=lib.mb_server_request_error(self._h, rid).decode())

    def result(self, rid: int):
        return self.out[rid]


def request_bytes(prob: inputs.Problem, precision=FP32) -> int:
    g, b, m, keep = _marshal(prob, precision)
    return int(lib.mb_request_bytes(ctypes.byref(g), ctypes.byref(b), ctypes.byref(m)))


BAND_DTYPE = np.dtype([("cell", "i4"), ("i", "i4"), ("j", "i4"), ("flags", "i4"),
                       ("aA", "f8"), ("aB", "f8"), ("aM", "f8"), ("bown", "f8"), ("d", "f8"),
                       ("nx", "f8"), ("ny", "f8"), ("wx", "f8"), ("wy", "f8"),
                       ("FB", "f8", 4), ("QB", "f8", 4), ("Qp", "f8", 4), ("Flo", "f8", 4), ("Fhi", "f8", 4),
                       ("C", "f8", 4), ("C2", "f8", 4), ("den", "f8"), ("mix", "i4"), ("aux", "i4"),
                       ("Flof", "f4", 4), ("Fhif", "f4", 4)])
assert BAND_DTYPE.itemsize == lib.mb_band_record_size(), "band record layout changed"
