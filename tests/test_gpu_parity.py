"""Parity of the CUDA sweep (through the C ABI) with the FP64 oracle on the
same seeded inputs: one sweep, several steps, batched instances, the
full-size single-instance workload, FP32 accuracy, conservation and the
degenerate cases.  Tolerances: FP64 contents alpha*Q to 1e-12 relative L-inf
per sweep; volume fractions to 1e-13; fluid/solid classes identical."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def mb():
    from paper_1711_11361_gb300 import mb as m
    return m


from gpu_util import compare, contents, rel_linf


def small_cases():
    return [
        ("cylinder_donor", inputs.small_case("cylinder", 48, 2.0)),
        ("cylinder_gcl", inputs.small_case("cylinder", 40, 2.5, uncover_mode=inputs.UNCOVER_FLUX_GCL)),
        ("triangle", inputs.small_case("triangle", 56, 1.7)),
        ("piston", inputs.small_case("piston", 72)),
        ("naca", inputs.c3_naca(96)),
        ("channel", inputs.c1_advection(60)),
    ]


@pytest.mark.parametrize("name,prob", small_cases(), ids=[c[0] for c in small_cases()])
def test_one_step_parity(mb, name, prob):
    orc = oracle.Oracle(prob)
    sim = mb.Sim(prob, mb.FP64)
    r0 = compare(sim, orc)
    assert r0["alpha"] <= 1e-13 and r0["cls"] == 0
    dt = orc.cfl_dt()
    for d in (0, 1):
        assert orc.sweep(d, dt) == 0
        sim.sweep(d, dt)
        r = compare(sim, orc)
        assert r["cls"] == 0, (name, d, r)
        assert r["alpha"] <= 1e-13, (name, d, r["alpha"])
        assert r["contents"] <= 1e-12, (name, d, r["contents"])


@pytest.mark.parametrize("name,prob", small_cases()[:4], ids=[c[0] for c in small_cases()[:4]])
def test_multi_step_parity(mb, name, prob):
    """Each step starts from the oracle's state (the one-step error is
    isolated, as round-off in tiny cut cells is amplified by 1/alpha from one
    step to the next); a second, free-running copy shows no drift."""
    orc = oracle.Oracle(prob)
    sim = mb.Sim(prob, mb.FP64)
    free = mb.Sim(prob, mb.FP64)
    worst, worst_free = 0.0, 0.0
    for k in range(12):
        clk = orc.clock()
        sim.write_state(0, orc.state(), clk["t"])
        dt = orc.cfl_dt()
        assert orc.step(dt)[0] == 0
        # the reseeded copy restarts its Strang alternation; keep its order equal
        if k % 2 == 1:
            sim.sweep(1, dt)
            sim.sweep(0, dt)
        else:
            sim.step(dt)
        free.step(dt)
        r = compare(sim, orc)
        assert r["cls"] == 0, (name, k)
        worst = max(worst, r["contents"])
        worst_free = max(worst_free, compare(free, orc)["contents"])
    assert worst <= 1e-12, (name, worst)
    assert worst_free <= 1e-9, (name, worst_free)


def test_device_cfl_matches_oracle(mb):
    prob = inputs.small_case("triangle", 64, 2.2)
    orc = oracle.Oracle(prob)
    sim = mb.Sim(prob, mb.FP64)
    for _ in range(3):
        r, dt_o = orc.step()
        dt_g = sim.step(0.0, report=True)[0]
        assert abs(dt_g - dt_o) <= 1e-14 * dt_o
    assert compare(sim, orc)["contents"] <= 1e-11


def test_batched_instances_match_oracle_and_solo(mb):
    probs = inputs.c4_batch(n=6, nmin=40, nmax=72, seed=7)
    sim = mb.Sim(probs, mb.FP64)
    orcs = [oracle.Oracle(p) for p in probs]
    solo = mb.Sim(probs[2], mb.FP64)
    dt = min(o.cfl_dt() for o in orcs)
    for k in range(6):
        for o in orcs:
            assert o.step(dt)[0] == 0
        sim.step(dt)
        solo.step(dt)
    for i, o in enumerate(orcs):
        r = compare(sim, o, i)
        assert r["cls"] == 0 and r["contents"] <= 1e-11, (i, probs[i].name, r["contents"])
    a = sim.read_state(2)["Q"]
    b = solo.read_state(0)["Q"]
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.nanmax(np.abs(a - b)) == 0.0


def test_graph_replay_equals_step_by_step(mb):
    prob = inputs.small_case("cylinder", 64, 2.0)
    s1 = mb.Sim(prob, mb.FP64)
    s2 = mb.Sim(prob, mb.FP64)
    for _ in range(7):
        s1.step(0.0)
    s2.run(7, 0.0)
    s2.sync()
    a, b = s1.read_state(0), s2.read_state(0)
    assert a["t"] == b["t"]
    assert np.array_equal(np.nan_to_num(a["Q"], nan=7.0), np.nan_to_num(b["Q"], nan=7.0))


def test_full_size_cylinder_parity(mb):
    """The 400x400 cylinder workload at its full size, a few steps, whole field."""
    prob = inputs.c2_cylinder(400)
    orc = oracle.Oracle(prob)
    sim = mb.Sim(prob, mb.FP64)
    for k in range(2):
        dt = orc.cfl_dt()
        orc.step(dt)
        sim.step(dt)
    r = compare(sim, orc)
    assert r["cls"] == 0 and r["contents"] <= 1e-11, r["contents"]


def test_full_size_pitching_naca_parity(mb):
    """The 1024x1024 pitching NACA 0012 workload at its full size, first 20
    steps free-running (each side at its own CFL step, which agree to
    round-off), whole field: contents to 1e-9, volume fractions to 1e-12,
    classes identical.  The FP32 form of the same run stays within 1e-4
    (L1 density, alpha-weighted) of the FP64 GPU path."""
    prob = inputs.c3_naca(1024)
    orc = oracle.Oracle(prob)
    sim = mb.Sim(prob, mb.FP64)
    s32 = mb.Sim(prob, mb.FP32)
    for k in range(20):
        assert orc.step()[0] == 0
        sim.step(0.0)
        s32.step(0.0)
    r = compare(sim, orc)
    assert r["cls"] == 0, r["cls"]
    assert r["alpha"] <= 1e-12, r["alpha"]
    assert r["contents"] <= 1e-9, r["contents"]
    g64, g32 = r["g"], s32.read_state(0)
    a = g64["alpha"]
    fl = a > 0
    l1 = np.sum(a[fl] * np.abs(g32["Q"][0][fl] - g64["Q"][0][fl])) / np.sum(a[fl] * g64["Q"][0][fl])
    assert l1 <= 1e-4, l1


def test_fp32_bulk_accuracy(mb):
    """FP32 bulk arithmetic with FP64 geometry and weights: L1 density error
    against the FP64 path stays below 1e-4 relative."""
    prob = inputs.c2_cylinder(200)
    s64 = mb.Sim(prob, mb.FP64)
    s32 = mb.Sim(prob, mb.FP32)
    for _ in range(60):
        dt = s64.step(0.0, report=True)[0]
        s32.step(dt)
    a = s64.read_state(0, alpha=True)
    b = s32.read_state(0)
    al = a["alpha"]
    fl = al > 0
    err = np.sum(al[fl] * np.abs(b["Q"][0][fl] - a["Q"][0][fl])) / np.sum(al[fl] * np.abs(a["Q"][0][fl]))
    assert err < 1e-4, err


@pytest.mark.parametrize("mode", [inputs.UNCOVER_DONOR, inputs.UNCOVER_FLUX_GCL])
def test_gpu_contents_change_only_by_wall_terms(mb, mode):
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_method import periodic_body_problem
    prob = periodic_body_problem("triangle", 48, (-0.3, 0.55), mode, state="bumpy")
    sim = mb.Sim(prob, mb.FP64)
    dt = oracle.Oracle(prob).cfl_dt()
    def tot():
        g = sim.read_state(0, alpha=True)
        return contents(g["Q"], g["alpha"]).sum(axis=(1, 2))
    scale = np.abs(tot()).max()
    for k in range(10):
        for d in ((0, 1) if k % 2 == 0 else (1, 0)):
            c0 = tot()
            sim.sweep(d, dt)
            w = sim.diagnostics(0)["wall"]
            assert np.max(np.abs(tot() - c0 - w)) / scale < 1e-13


def test_degenerate_cases(mb):
    # no body at all
    p = inputs.Problem("empty", 16, 12, 0.0, 0.0, 1.0, 0.75, bc=(1, 1, 0, 0))
    X, Y = p.cell_centres()
    p.Q0 = inputs.conserved(1.0 + 0.2 * np.sin(2 * np.pi * X), 0.1, 0.0, 1.0)
    o, s = oracle.Oracle(p), mb.Sim(p, mb.FP64)
    for _ in range(3):
        dt = o.cfl_dt()
        o.step(dt)
        s.step(dt)
    assert compare(s, o)["contents"] <= 1e-12
    # body entirely outside the domain, minimum grid size
    p2 = inputs.Problem("outside", 8, 8, 0.0, 0.0, 1.0, 1.0, polygons=[inputs.triangle_polygon(3.0, 3.0, 0.5)],
                        moving=[1], U=(0.3, 0.0))
    p2.Q0 = inputs.conserved(np.ones((8, 8)), 0.0, 0.0, 1.0)
    s2 = mb.Sim(p2, mb.FP64)
    s2.step(0.0)
    assert np.allclose(s2.read_state(0)["Q"][0], 1.0, atol=0, rtol=1e-15)
    # invalid arguments fail loudly
    bad = inputs.Problem("bad", 4, 4, 0.0, 0.0, 1.0, 1.0)
    with pytest.raises(mb.MBError):
        mb.Sim(bad, mb.FP64)
