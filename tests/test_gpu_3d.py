"""The three-dimensional CUDA path (include/mb3.h) against the three-
dimensional oracle (itself pinned to closed forms and to the two-dimensional
oracle in tests/test_oracle_3d.py), through the C ABI: volume fractions at a
pose, one sweep along each axis from identical input in both uncovering
modes, whole steps re-seeded from the oracle, the CFL step, uniform flow, a
cone meeting a shock free running, and the Schardin workload itself (a small
mesh free running, and the bench's 20-cells-per-D mesh sweep by sweep).
Tolerances: contents alpha*Q to 1e-12 relative per sweep from identical
input; after a second and third sweep, round-off in a cut cell's content
divided by its volume fraction enters the fluxes, as in two dimensions."""
import math

import numpy as np
import pytest

from oracle import o3
from paper_1711_11361_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def mb3():
    from paper_1711_11361_gb300 import mb3 as m
    return m


def _rel(a, b):
    """max over components of max|a - b| / max|b| (a zero component against
    1e-2 of the largest component's scale)"""
    big = max(np.max(np.abs(b[q])) for q in range(b.shape[0]))
    return max(np.max(np.abs(a[q] - b[q])) / max(np.max(np.abs(b[q])), 1e-2 * big) for q in range(b.shape[0]))


def _cone(nx=24, uniform=False, U=(0.35, 0.12, -0.08), mode=inputs.UNCOVER_DONOR, bc=(inputs.PERIODIC,) * 6):
    n, c, bb = inputs.cone_planes((0.63, 0.5123, 0.4871), 0.35, 0.2, 12)
    p = inputs.Problem3("cone", nx, nx, nx, normals=n, offsets=c, bbox=bb, U=U, bc=bc, uncover_mode=mode)
    X, Y, Z = p.cell_centres()
    if uniform:
        p.Q0 = inputs.conserved3(np.ones_like(X), U[0], U[1], U[2], np.ones_like(X))
    else:
        tp = 2 * math.pi
        p.Q0 = inputs.conserved3(1 + 0.2 * np.sin(tp * X) * np.cos(tp * Y), U[0] + 0.1 * np.sin(tp * Z), U[1],
                                 U[2] + 0.05 * np.cos(tp * X), 1 + 0.1 * np.cos(tp * (X + Z)))
    return p


def test_volume_fractions_at_a_pose(mb3):
    p = _cone(nx=32)
    T = (0.0123, -0.0311, 0.0277)
    sim = mb3.Sim3(p, write_initial=False)
    sim.write_state(p.Q0, 0.0, T)
    a_gpu = sim.read_state(alpha=True)["alpha"]
    a_orc, _, _ = o3.Oracle3(p).geometry(T)
    assert np.max(np.abs(a_gpu - a_orc)) < 1e-13
    assert np.sum((a_orc > 0) & (a_orc < 1)) > 100
    sim.close()


@pytest.mark.parametrize("mode", [inputs.UNCOVER_DONOR, inputs.UNCOVER_FLUX_GCL])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_one_sweep_from_identical_input(mb3, d, mode):
    p = _cone(mode=mode)
    orc = o3.Oracle3(p)
    sim = mb3.Sim3(p)
    dt = orc.cfl_dt()
    for _ in range(2):   # a few steps first, so that the body has cut cells of every kind
        orc.step(dt)
    clk = orc.clock()
    sim.write_state(orc.state(), clk["t"], clk["T"])
    orc.set_state(orc.state(), clk["t"], clk["T"], 0)
    assert orc.sweep(d, dt) == 0
    sim.sweep(d, dt)
    assert _rel(sim.contents(), orc.contents()) <= 1e-12
    wo, mo = orc.last_sweep()
    wg, mg = sim.last_sweep()
    assert mg == mo
    assert np.max(np.abs(wg - wo)) <= 1e-12 * max(1.0, np.max(np.abs(wo)))
    sim.close()


@pytest.mark.parametrize("mode", [inputs.UNCOVER_DONOR, inputs.UNCOVER_FLUX_GCL])
def test_steps_reseeded_from_the_oracle(mb3, mode):
    """Six steps, each from the oracle's state (x, y, z then z, y, x): the
    first sweep of a step to 1e-11 (the two sides compute volumes by
    different algorithms, which agree to about 1e-13, and the small
    w-momentum component is measured on its own scale; the tighter one-sweep
    test above holds 1e-12).  A later sweep starts from contents
    already round-off apart; in a cut cell of volume fraction alpha that
    difference becomes difference/alpha in its state and reaches the next
    sweep's fluxes, once per sweep: after m sweeps the bound is 1e-15 over
    the product of the earlier sweeps' smallest volume fractions (at least
    1e-11)."""
    p = _cone(mode=mode)
    orc = o3.Oracle3(p)
    sim = mb3.Sim3(p)
    for s in range(6):
        clk = orc.clock()
        sim.write_state(orc.state(), clk["t"], clk["T"])
        orc.set_state(orc.state(), clk["t"], clk["T"], s)
        dt = orc.cfl_dt()
        assert abs(sim.cfl_dt() - dt) <= 1e-14 * dt
        order = (0, 1, 2) if s % 2 == 0 else (2, 1, 0)
        amp = 1.0
        for m, d in enumerate(order):
            assert orc.sweep(d, dt) == 0
            sim.sweep(d, dt)
            tol = 1e-11 if m == 0 else max(1e-11, 1e-15 / amp)
            assert _rel(sim.contents(), orc.contents()) <= tol, (s, d)
            a = orc.alpha()
            amp *= a[a > 0].min()
    sim.close()


def test_uniform_flow_with_the_cone_stays_uniform(mb3):
    p = _cone(uniform=True, mode=inputs.UNCOVER_FLUX_GCL)
    sim = mb3.Sim3(p)
    for _ in range(4):
        sim.step()
    s = sim.read_state(alpha=True)
    Q, a = s["Q"], s["alpha"]
    E = 1.0 / 0.4 + 0.5 * (0.35 ** 2 + 0.12 ** 2 + 0.08 ** 2)
    fl = a > 0
    for q, v in enumerate((1.0, 0.35, 0.12, -0.08, E)):
        assert np.max(a[fl] * np.abs(Q[q][fl] - v)) < 1e-8
    sim.close()


def test_cone_meets_a_shock_free_running(mb3):
    """A cone moving with the gas into a Mach-1.5 shock (transmissive box):
    10 free-running steps at the device's CFL step, each oracle step at the
    device's dt; contents to 1e-9."""
    n, c, bb = inputs.cone_planes((0.45, 0.5123, 0.4871), 0.3, 0.17, 12)
    U = (0.5 * math.sqrt(1.4), 0.0, 0.0)
    p = inputs.Problem3("cone_shock", 32, 24, 24, normals=n, offsets=c, bbox=bb, U=U)
    X, Y, Z = p.cell_centres()
    r2, u2, p2 = inputs.post_shock(1.5)
    right = X > 0.6
    p.Q0 = inputs.conserved3(np.where(right, r2, 1.0), np.where(right, U[0] + u2, U[0]), 0.0, 0.0,
                             np.where(right, p2, 1.0))
    orc = o3.Oracle3(p)
    sim = mb3.Sim3(p)
    for _ in range(10):
        dt = sim.step()
        assert orc.step(dt)[0] == 0
    assert _rel(sim.contents(), orc.contents()) <= 1e-9
    assert sim.read_state()["step"] == 10
    sim.close()


def test_schardin_cone_small_mesh_free_running(mb3):
    """The Schardin workload (inputs.n3_schardin_cone) at 4 cells per D (40 x
    40 x 20): the cone on the reflective side z = 0, the stationary shock,
    transmissive sides; 12 free-running steps at the device's dt, each
    oracle step at that dt; contents to 1e-9 relative."""
    p = inputs.n3_schardin_cone(4)
    orc = o3.Oracle3(p)
    sim = mb3.Sim3(p)
    for _ in range(12):
        dt = sim.step()
        assert orc.step(dt)[0] == 0
    assert _rel(sim.contents(), orc.contents()) <= 1e-9
    assert sim.last_sweep()[1] == orc.last_sweep()[1]
    assert sim.read_state()["status"] == 0
    sim.close()


def test_schardin_cone_bench_mesh_sweeps(mb3):
    """The bench's 20-cells-per-D mesh (200 x 200 x 100, 4 M cells, the
    launch configuration bench.py times), the shock moved 0.4 D behind the
    apex so that it crosses the cone's surface: two steps, each started from
    the oracle's state, every sweep compared as in the re-seeded test."""
    p = inputs.n3_schardin_cone(20)
    X, Y, Z = p.cell_centres()
    r2, u2, p2 = p.info["post_shock"]
    xs = p.info["shock_x"] - 2.0 / 20 - 0.4
    right = X > xs
    p.Q0 = inputs.conserved3(np.where(right, r2, 1.0), np.where(right, u2, p.info["u1"]), 0.0, 0.0,
                             np.where(right, p2, 1.0))
    orc = o3.Oracle3(p)
    sim = mb3.Sim3(p)
    for s in range(2):
        clk = orc.clock()
        sim.write_state(orc.state(), clk["t"], clk["T"])
        orc.set_state(orc.state(), clk["t"], clk["T"], s)
        dt = orc.cfl_dt()
        assert abs(sim.cfl_dt() - dt) <= 1e-14 * dt
        amp = 1.0
        for m, d in enumerate((0, 1, 2) if s % 2 == 0 else (2, 1, 0)):
            assert orc.sweep(d, dt) == 0
            sim.sweep(d, dt)
            tol = 1e-11 if m == 0 else max(1e-11, 1e-15 / amp)
            assert _rel(sim.contents(), orc.contents()) <= tol, (s, d)
            assert sim.last_sweep()[1] == orc.last_sweep()[1]
            a = orc.alpha()
            amp *= a[a > 0].min()
    sim.close()


def _l1_rel(a, b, w):
    return float(np.sum(w * np.abs(a - b)) / np.sum(w * np.abs(b)))


def test_fp32_flux_option_tracks_the_fp64_path(mb3):
    """mb3_set_precision(MB_FP32) evolves and solves the Riemann problems of
    faces without a wall part in FP32 from an FP32 copy of the state. On the
    cone-and-shock case with the FP64 path's dt every step (20 steps): the
    alpha-weighted L1 density difference against the FP64 path (held to the
    oracle above) at most 1e-4, the FP32 path's stated accuracy bar, and the
    same step count and status."""
    from paper_1711_11361_gb300 import mb
    n, c, bb = inputs.cone_planes((0.45, 0.5123, 0.4871), 0.3, 0.17, 12)
    U = (0.5 * math.sqrt(1.4), 0.0, 0.0)
    p = inputs.Problem3("cone_shock", 32, 24, 24, normals=n, offsets=c, bbox=bb, U=U)
    X, Y, Z = p.cell_centres()
    r2, u2, p2 = inputs.post_shock(1.5)
    right = X > 0.6
    p.Q0 = inputs.conserved3(np.where(right, r2, 1.0), np.where(right, U[0] + u2, U[0]), 0.0, 0.0,
                             np.where(right, p2, 1.0))
    s64 = mb3.Sim3(p)
    s32 = mb3.Sim3(p, precision=mb.FP32)
    for _ in range(20):
        dt = s64.step()
        s32.step(dt)
    a = s64.read_state(alpha=True)
    b = s32.read_state(alpha=True)
    fl = a["alpha"] > 0
    assert np.array_equal(fl, b["alpha"] > 0)
    err = _l1_rel(b["Q"][0][fl], a["Q"][0][fl], a["alpha"][fl])
    assert 0.0 < err <= 1e-4, err
    assert a["status"] == 0 and b["status"] == 0 and b["step"] == 20
    s64.close()
    s32.close()


def test_fp32_flux_option_conserves_like_fp64(mb3):
    """Closed periodic box, FP32 flux option: fluxes are stored in FP64 and
    the update runs in FP64, so per sweep the total contents change only by
    the reported wall terms, to 1e-12 as in the FP64 path."""
    from paper_1711_11361_gb300 import mb
    p = _cone(mode=inputs.UNCOVER_FLUX_GCL)
    sim = mb3.Sim3(p, precision=mb.FP32)
    dt = sim.cfl_dt()
    for d in (0, 1, 2, 2, 1, 0):
        c0 = sim.contents().sum(axis=(1, 2, 3))
        sim.sweep(d, dt)
        c1 = sim.contents().sum(axis=(1, 2, 3))
        w, _ = sim.last_sweep()
        assert np.max(np.abs(c1 - c0 - w)) < 1e-12 * max(1.0, np.max(np.abs(c0)))
    sim.close()


def test_fp32_flux_option_keeps_uniform_flow(mb3):
    """Gas moving with the cone, FP32 flux option: uniform to FP32 rounding
    (alpha-weighted deviation below 1e-5 after four steps)."""
    from paper_1711_11361_gb300 import mb
    p = _cone(uniform=True, mode=inputs.UNCOVER_FLUX_GCL)
    sim = mb3.Sim3(p, precision=mb.FP32)
    for _ in range(4):
        sim.step()
    s = sim.read_state(alpha=True)
    Q, a = s["Q"], s["alpha"]
    E = 1.0 / 0.4 + 0.5 * (0.35 ** 2 + 0.12 ** 2 + 0.08 ** 2)
    fl = a > 0
    for q, v in enumerate((1.0, 0.35, 0.12, -0.08, E)):
        assert np.max(a[fl] * np.abs(Q[q][fl] - v)) < 1e-5
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_schardin_cone_finest_mesh_conserves(mb3, precision):
    """The bench's finest mesh (40 cells per D, 400 x 400 x 200, 32 M cells,
    the launch configuration bench.py times), where the oracle is too slow
    to run: a property that holds at any size.  Per sweep of the first two
    steps the total contents change by the reported wall terms alone: the
    shock is stationary, so the fluxes through the open x sides are the same
    Rankine-Hugoniot flux, and the open y sides pass equal pressures.  The
    one exception is the z momentum in a z sweep, which also takes the
    pressure on the symmetry plane z = 0 where the cone's section covers it
    (the three-dimensional oracle shows the same at 4 and 8 cells per D).
    To 1e-11 of the largest total (fluxes are stored and the update runs in
    FP64 in both precisions).  With the FP32 flux option the two x-side
    fluxes are FP32 values of states whose exact fluxes are equal, so an x
    sweep may also differ by their rounding, the same at every face pair:
    at most 16 roundings of 2^-24 each (the flux's chain of operations) of
    the largest flux component on either side, times dt/h and the ny nz
    face pairs."""
    from paper_1711_11361_gb300 import mb
    p = inputs.n3_schardin_cone(40)
    sim = mb3.Sim3(p, precision=mb.FP32 if precision == "fp32" else mb.FP64)
    dt = sim.cfl_dt()
    r2, u2, p2 = p.info["post_shock"]
    u1, g = p.info["u1"], p.gamma

    def fx(r, u, pr):   # the x flux of a uniform state at rest in y and z
        return max(abs(r * u), abs(r * u * u + pr), abs(u * (pr / (g - 1.0) + 0.5 * r * u * u + pr)))
    fmax = max(fx(1.0, u1, 1.0), fx(r2, u2, p2))
    c0 = sim.contents().sum(axis=(1, 2, 3))
    scale = np.abs(c0).max()
    for d in (0, 1, 2, 2, 1, 0):
        sim.sweep(d, dt)
        c1 = sim.contents().sum(axis=(1, 2, 3))
        w, _ = sim.last_sweep()
        q = [0, 1, 2, 4] if d == 2 else [0, 1, 2, 3, 4]
        tol = 1e-11 * scale
        if precision == "fp32" and d == 0:
            tol += 2.0 * 16 * 2.0 ** -24 * fmax * dt / p.h[0] * p.ny * p.nz
        assert np.max(np.abs((c1 - c0 - w)[q])) <= tol, (d, c1 - c0 - w)
        c0 = c1
    assert sim.read_state()["status"] == 0
    sim.close()


def test_no_body_shock_tube_along_each_axis(mb3):
    """No body (an empty region R: the geometry, wall and event kernels do
    not run): a shock tube along x, y and z in turn, with the tangential
    velocities nonzero, 8 free-running steps against the oracle at the
    device's dt; contents to 1e-11 relative (no cut cells, so no 1/alpha
    growth of round-off)"""
    for d in range(3):
        p = inputs.Problem3("tube", 24, 20, 16, hi=(1.2, 1.0, 0.8))
        c = p.cell_centres()[d]
        hi = (1.2, 1.0, 0.8)[d]
        left = c < 0.45 * hi
        vel = [np.full_like(c, 0.2), np.full_like(c, -0.1), np.full_like(c, 0.05)]
        vel[d] = np.zeros_like(c)
        p.Q0 = inputs.conserved3(np.where(left, 1.0, 0.125), vel[0], vel[1], vel[2], np.where(left, 1.0, 0.1))
        orc = o3.Oracle3(p)
        sim = mb3.Sim3(p)
        for _ in range(8):
            dt = sim.step()
            assert orc.step(dt)[0] == 0
        assert _rel(sim.contents(), orc.contents()) <= 1e-11, d
        assert sim.read_state()["status"] == 0
        sim.close()


def test_many_collapse_seeds_take_the_one_thread_merge(mb3):
    """A box body whose front face crosses a layer of identical cells: in
    the first x sweep every cell of that layer keeps under 1% of its volume
    (alpha 0.5 -> 0.004), so several hundred collapse seeds merge at once,
    more than the block-wide merge holds (146 seeds), and the one-thread
    form runs.  Contents to 1e-12 and the same merged-cell count as the
    oracle (940 cells)."""
    h = 1.0 / 32
    N = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], float)
    lo, hi = (0.2, 0.2031, 0.2017), (16.5 * h, 0.7969, 0.7983)
    C = np.array([-lo[0], hi[0], -lo[1], hi[1], -lo[2], hi[2]])
    U = 2.0
    p = inputs.Problem3("slab3", 32, 32, 32, normals=N, offsets=C, bbox=(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]),
                        U=(U, 0.0, 0.0), bc=(inputs.PERIODIC,) * 6)
    X, Y, Z = p.cell_centres()
    p.Q0 = inputs.conserved3(np.ones_like(X), 0.0, 0.0, 0.0, np.ones_like(X))
    orc = o3.Oracle3(p)
    sim = mb3.Sim3(p)
    dt = 0.496 * h / U
    assert orc.sweep(0, dt) == 0
    sim.sweep(0, dt)
    _, mo = orc.last_sweep()
    _, mg = sim.last_sweep()
    assert mo > 146 and mg == mo
    assert _rel(sim.contents(), orc.contents()) <= 1e-12
    sim.close()
