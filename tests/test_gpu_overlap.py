"""The FP32 Euler sweep split into two bulk passes (the cells that need no
band data, run concurrently with the geometry and band-flux kernels, then
the deferred cells near the body) gives the same bits as every cell waiting
for the band fluxes, for translating, static and rotating bodies (a
rotating body's cells all take the second pass), through CUDA-graph replay
and step by step."""
import numpy as np
import pytest

from paper_1711_11361_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def mb():
    from paper_1711_11361_gb300 import mb as m
    return m


def _mix():
    return [
        inputs.small_case("cylinder", 48, 2.0),
        inputs.small_case("triangle", 56, 1.7),
        inputs.small_case("piston", 64),
        inputs.small_case("cylinder", 130, 1.4),
        inputs.small_case("triangle", 200, 2.6),
        inputs.small_case("piston", 150),
        inputs.c3_naca(128),
    ]


def _run(mb, probs, overlap, steps, graphs=True, dt=0.0):
    sim = mb.Sim(probs, mb.FP32)
    sim.set_overlap(overlap)
    if graphs:
        sim.run(steps, dt)
    else:
        for _ in range(steps):
            sim.step(dt)
    out = [sim.read_state(k)["Q"] for k in range(len(probs))]
    sim.close()
    return out


def test_two_pass_equals_one_pass(mb):
    probs = _mix()
    a = _run(mb, probs, True, 25)
    b = _run(mb, probs, False, 25)
    for k, p in enumerate(probs):
        assert np.array_equal(a[k], b[k], equal_nan=True), p.name


def test_two_pass_step_by_step_equals_graph(mb):
    probs = _mix()[:4]
    a = _run(mb, probs, True, 8, graphs=True)
    b = _run(mb, probs, True, 8, graphs=False)
    for k, p in enumerate(probs):
        assert np.array_equal(a[k], b[k], equal_nan=True), p.name
