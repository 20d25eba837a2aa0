"""Dynamic batches and the continuous-batching request loop on the GPU:
instances added to and removed from a running batch keep evolving exactly
as they would alone, and every request served through mb_server_* returns
the same state (bit for bit) as the same simulation run alone, whatever the
mix it ran in, the order of arrival and the memory budget."""
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
        inputs.small_case("cylinder", 40, 1.4),
        inputs.small_case("triangle", 72, 2.6),
        inputs.small_case("piston", 48),
    ]


def _solo(mb, prob, nsteps, precision):
    sim = mb.Sim(prob, precision)
    sim.run(nsteps, 0.0)
    out = sim.read_state(0)
    sim.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_add_remove_matches_solo(mb, precision):
    prec = mb.FP64 if precision == "fp64" else mb.FP32
    probs = _mix()[:4]
    sim = mb.Sim(probs[:2], prec)
    sim.run(2, 0.0)                      # instances 0, 1: 2 steps
    k = sim.add(probs[2])                # joins at an even batch step
    assert k == 2
    sim.run(4, 0.0)                      # 0, 1: 6 steps; 2: 4 steps
    sim.remove(0)                        # 1 -> 0, 2 -> 1
    k = sim.add(probs[3])                # 3 joins as index 2
    sim.run(2, 0.0)                      # old 1: 8, old 2: 6, new: 2
    got = [sim.read_state(i) for i in range(3)]
    want = [(probs[1], 8), (probs[2], 6), (probs[3], 2)]
    for g, (p, n) in zip(got, want):
        s = _solo(mb, p, n, prec)
        assert g["step"] == n
        assert np.array_equal(g["Q"], s["Q"], equal_nan=True), p.name
        assert g["t"] == s["t"]


def test_server_results_equal_solo_in_any_mix(mb):
    probs = _mix()
    steps = [12, 7, 20, 9, 15, 6, 11, 8]
    reqs = [(probs[k % len(probs)], steps[k]) for k in range(8)]
    srv = mb.Server(mb.FP32, 0, budget_bytes=2 ** 34, max_active=3)
    ids, peak, ticks = [], 0, 0
    # staggered arrivals: two requests, then one more every third tick
    ids.append(srv.submit(*reqs[0]))
    ids.append(srv.submit(*reqs[1]))
    nxt = 2
    admitted_while_running = False
    while True:
        before = sum(srv.query(i)["state"] == mb.Server.RUNNING for i in ids)
        a, q, d = srv.tick()
        ticks += 1
        peak = max(peak, a)
        if before > 0 and a > before:
            admitted_while_running = True
        if nxt < len(reqs) and ticks % 3 == 0:
            ids.append(srv.submit(*reqs[nxt]))
            nxt += 1
        if nxt == len(reqs) and d == len(reqs):
            break
        assert ticks < 500
    assert peak >= 2 and admitted_while_running
    for rid, (p, n) in zip(ids, reqs):
        info = srv.query(rid)
        assert info["state"] == mb.Server.DONE and info["steps"] == n
        assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
        s = _solo(mb, p, n, mb.FP32)
        assert np.array_equal(srv.result(rid), s["Q"], equal_nan=True), (rid, p.name)
    srv.close()


def test_server_admits_by_memory_budget(mb):
    probs = _mix()[:3]
    # no two requests fit together (a request above the budget runs alone)
    need = min(mb.request_bytes(p, mb.FP32) for p in probs)
    srv = mb.Server(mb.FP32, 0, budget_bytes=1.5 * need, max_active=8)
    ids = [srv.submit(p, 5) for p in probs]
    peak = 0
    for _ in range(100):
        a, q, d = srv.tick()
        peak = max(peak, a)
        if d == len(ids):
            break
    assert peak == 1                      # one request at a time fits the budget
    for rid, p in zip(ids, probs):
        assert srv.query(rid)["state"] == mb.Server.DONE
        assert np.array_equal(srv.result(rid), _solo(mb, p, 5, mb.FP32)["Q"], equal_nan=True)
    srv.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_changes_no_result(mb, precision):
    """Launch shapes picked by mb_autotune (CTA sizes, rows per thread of
    the y sweep) move work between threads only: the state is bit-identical
    to an untuned run, and tuning in mid-run changes nothing."""
    prec = mb.FP64 if precision == "fp64" else mb.FP32
    probs = _mix()[:3]
    a = mb.Sim(probs, prec)
    a.run(3, 0.0)
    choice = a.autotune()
    assert choice["x_cta"] in (64, 128, 256) and choice["y_rows"] in (32, 64, 128)
    a.run(3, 0.0)
    b = mb.Sim(probs, prec)
    b.run(6, 0.0)
    for k in range(len(probs)):
        assert np.array_equal(a.read_state(k)["Q"], b.read_state(k)["Q"], equal_nan=True), k
