"""The positivity safeguard on the GPU (cluster mixing of non-physical cells
and of cells that keep less than 1% of their volume over a sweep with their
fluid face neighbours, a reading: the paper gives none) against the oracle:
- a triangle on 751^2, shock Mach 1.918, from the seeded 64-instance batch,
  whose corners leave slivers in most x sweeps (the oracle merges cells in
  the x sweeps of steps 56 and 57);
- a slab whose front face covers a column from 0.3 to 0.002 of its volume in
  one x sweep (every cell of that column seeds a merge)."""
import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

from gpu_util import compare


@pytest.fixture(scope="module")
def mb():
    from paper_1711_11361_gb300 import mb as m
    return m


def test_safeguard_merges_like_oracle(mb):
    prob = inputs.c4_batch()[60]
    assert prob.name.startswith("c4_60_triangle_N751")
    orc = oracle.Oracle(prob)
    for _ in range(56):
        assert orc.step()[0] == 0
    sim = mb.Sim(prob, mb.FP64)
    merged = []
    for k in (56, 57):
        clk = orc.clock()
        sim.write_state(0, orc.state(), clk["t"])
        dt = orc.cfl_dt()
        order = (0, 1) if k % 2 == 0 else (1, 0)
        # first sweep from the oracle's state: contents to 1e-12.  Second
        # sweep: the first sweep's round-off in the smallest cut cells is
        # divided by alpha (down to ~1e-6 here) when their states Q = C/alpha
        # are formed and enters the second sweep's fluxes: 1e-10.
        for d, tol in zip(order, (1e-12, 1e-10)):
            assert orc.sweep(d, dt) == 0
            sim.sweep(d, dt)
            mo, mg = orc.last_sweep()[1], sim.diagnostics()["mixed"]
            assert mg == mo, (k, d, mg, mo)
            merged.append(mg)
            r = compare(sim, orc)
            assert r["cls"] == 0, (k, d)
            assert r["contents"] <= tol, (k, d, r["contents"])
    assert merged[0] > 0 and merged[3] > 0, merged


def test_fp32_batch_long_run_stays_physical(mb):
    """The 64-instance FP32 batch for 120 steps at the CFL step: every
    non-physical cell is merged and no instance reports an error."""
    probs = inputs.c4_batch()
    sim = mb.Sim(probs, mb.FP32)
    sim.run(120, 0.0)
    assert sim.sync() == 0
    for k in range(len(probs)):
        assert sim.read_state(k)["step"] == 120


def test_collapse_merges_like_oracle(mb):
    """One x sweep of the collapsing slab (see tests/test_oracle_pins.py) from
    a non-uniform state: the GPU's FP64 contents equal the oracle's to 1e-12
    and both merge the same cells."""
    prob = inputs.collapse_slab(uniform=False)
    orc = oracle.Oracle(prob)
    sim = mb.Sim(prob, mb.FP64)
    sim.write_state(0, orc.state(), 0.0)
    dt = inputs.COLLAPSE_SLAB_DT
    assert orc.sweep(0, dt) == 0
    sim.sweep(0, dt)
    mo, mg = orc.last_sweep()[1], sim.diagnostics()["mixed"]
    assert mo > 0 and mg == mo, (mg, mo)
    r = compare(sim, orc)
    assert r["cls"] == 0
    assert r["contents"] <= 1e-12, r["contents"]
