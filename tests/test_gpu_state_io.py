"""Batched host state I/O (mb_write_states / mb_read_states): the same bits as
one mb_write_state / mb_read_state call per instance, whether the host
arrays are pageable or page-locked, in FP32 and FP64; a write followed by
a read returns the state rounded to the batch's precision, NaN in solid
cells."""
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
        inputs.small_case("triangle", 150, 1.7),
        inputs.small_case("piston", 64),
        inputs.small_case("cylinder", 200, 1.4),
        inputs.c3_naca(128),
    ]


def _pinned(arrays):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrays]


def _times(probs):
    return [0.0 if k % 2 == 0 else 0.003 * k for k in range(len(probs))]


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_batched_write_equals_per_instance(mb, prec):
    probs = _mix()
    P = getattr(mb, prec)
    ts = _times(probs)
    a = mb.Sim(probs, P, write_initial=False)
    for k, p in enumerate(probs):
        a.write_state(k, p.Q0, ts[k])
    b = mb.Sim(probs, P, write_initial=False)
    b.write_states([p.Q0 for p in probs], ts)
    c = mb.Sim(probs, P, write_initial=False)
    pin = _pinned([p.Q0 for p in probs])
    c.write_states([t.data_ptr() for t in pin], ts)
    for s in (a, b, c):
        s.run(6, 0.0)
    for k, p in enumerate(probs):
        ra, rb, rc = a.read_state(k), b.read_state(k), c.read_state(k)
        assert np.array_equal(ra["Q"], rb["Q"], equal_nan=True), p.name
        assert np.array_equal(ra["Q"], rc["Q"], equal_nan=True), p.name
        assert ra["t"] == rb["t"] == rc["t"] and ra["step"] == rb["step"] == rc["step"] == 6
    for s in (a, b, c):
        s.close()


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_batched_read_equals_per_instance(mb, prec):
    probs = _mix()
    sim = mb.Sim(probs, getattr(mb, prec))
    sim.run(5, 0.0)
    one = [sim.read_state(k) for k in range(len(probs))]
    pageable, clk, r = sim.read_states()
    assert r == 0
    pin = _pinned([np.zeros((p.nc, p.ny, p.nx)) for p in probs])
    _, clk2, r2 = sim.read_states([t.data_ptr() for t in pin])
    assert r2 == 0
    for k, p in enumerate(probs):
        assert np.array_equal(one[k]["Q"], pageable[k], equal_nan=True), p.name
        assert np.array_equal(one[k]["Q"], pin[k].numpy(), equal_nan=True), p.name
        assert clk[k, 0] == clk2[k, 0] == one[k]["t"]
        assert clk[k, 3] == one[k]["step"] == 5
    sim.close()


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_write_read_round_trip(mb, prec):
    probs = _mix()
    sim = mb.Sim(probs, getattr(mb, prec), write_initial=False)
    rng = np.random.default_rng(7)
    Qs = []
    for p in probs:
        Q = np.array(p.Q0, dtype=np.float64, copy=True)
        Q *= 1.0 + 1e-3 * rng.standard_normal(Q.shape)
        Qs.append(Q)
    pin = _pinned(Qs)
    sim.write_states([t.data_ptr() for t in pin])
    out, clk, r = sim.read_states()
    assert r == 0
    for k, p in enumerate(probs):
        a = sim.read_state(k, alpha=True)["alpha"]
        solid = a == 0.0
        want = Qs[k].astype(np.float32).astype(np.float64) if prec == "FP32" else Qs[k]
        assert np.all(np.isnan(out[k][:, solid])), p.name
        assert np.array_equal(out[k][:, ~solid], want[:, ~solid]), p.name
    sim.close()


def test_first_step_dt_is_the_fp64_one(mb):
    """The first step's wave speeds of a written FP32 state are the FP64
    maxima over the stored states, screened in FP32 without changing the
    result: with initial states that FP32 holds exactly, the FP32 and FP64
    batches take the same first CFL step, bit for bit."""
    probs = _mix()
    for p in probs:
        p.Q0 = np.asarray(p.Q0, dtype=np.float32).astype(np.float64)
    dts = []
    for prec in (mb.FP32, mb.FP64):
        sim = mb.Sim(probs, prec)
        dts.append(sim.step(0.0, report=True))
        sim.close()
    assert np.array_equal(dts[0], dts[1]), (dts[0], dts[1])


def test_fp32_host_io_matches_fp64_host_io(mb):
    """mb_write_states_f32 / mb_read_states_f32 on an FP32 batch: writing the
    FP32 roundings of the FP64 states gives the same device bits (and so the
    same steps) as writing the FP64 states, and the FP32 read returns the
    device values exactly (the FP64 read's values, rounded)."""
    probs = _mix()
    ts = _times(probs)
    a = mb.Sim(probs, mb.FP32, write_initial=False)
    a.write_states([p.Q0 for p in probs], ts)
    b = mb.Sim(probs, mb.FP32, write_initial=False)
    b.write_states([p.Q0.astype(np.float32) for p in probs], ts, dtype=np.float32)
    c = mb.Sim(probs, mb.FP32, write_initial=False)
    pin = _pinned([p.Q0.astype(np.float32) for p in probs])
    c.write_states([t.data_ptr() for t in pin], ts, dtype=np.float32)
    for s in (a, b, c):
        s.run(5, 0.0)
    qa, ca, _ = a.read_states()
    qb, cb, _ = b.read_states(dtype=np.float32)
    qc, cc, _ = c.read_states(dtype=np.float32)
    assert np.array_equal(ca, cb) and np.array_equal(ca, cc)
    for k, p in enumerate(probs):
        assert qb[k].dtype == np.float32
        assert np.array_equal(qa[k].astype(np.float32), qb[k], equal_nan=True), p.name
        assert np.array_equal(qb[k], qc[k], equal_nan=True), p.name
    for s in (a, b, c):
        s.close()


def test_fp32_host_io_on_fp64_batch(mb):
    """On an FP64 batch the FP32 host values are widened exactly on writing
    and rounded on reading."""
    probs = _mix()[:3]
    q32 = [p.Q0.astype(np.float32) for p in probs]
    s = mb.Sim(probs, mb.FP64, write_initial=False)
    s.write_states(q32, dtype=np.float32)
    q64, _, _ = s.read_states()
    q32b, _, _ = s.read_states(dtype=np.float32)
    for k in range(len(probs)):
        fl = np.isfinite(q64[k][0])
        assert np.array_equal(q64[k][:, fl], q32[k][:, fl].astype(np.float64))
        assert np.array_equal(q32b[k], q64[k].astype(np.float32), equal_nan=True)
    s.close()
