"""Host logic of bench.py's multi-rank (torchrun) path, run as two gloo ranks
on the CPU: each rank advances its own seeded batch of independent instances
(weak scaling, no collective on the data path), the whole-job time is the
slowest rank's and the whole-job cell count is the sum over ranks."""
import argparse
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = argparse.Namespace(workload="c4", instances=3)
        probs, name = bench.workload(rank, args)
        cells = sum(p.nx * p.ny for p in probs)
        fake_ms = 100.0 + 50.0 * rank
        total_ms, cells_all = bench.combine_ranks(fake_ms, cells, "cpu")
        q.put((rank, name, [p.name for p in probs], cells, total_ms, cells_all,
               bench.job_value(cells_all, 10, total_ms)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_combine():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, names0, c0, t0, ca0, v0), (r1, n1, names1, c1, t1, ca1, v1) = res
    assert n0 == n1
    # every rank has its own batch (independent instances), drawn from the same recipe
    assert names0 != names1
    assert len(names0) == len(names1) == 3
    # max over ranks of the timed region, sum over ranks of the work, same on every rank
    assert t0 == t1 == 150.0
    assert ca0 == ca1 == float(c0 + c1)
    assert v0 == v1 == pytest.approx((c0 + c1) * 2 * 10 / 0.150)


def test_single_process_passthrough():
    import bench
    assert bench.combine_ranks(12.5, 1000, "cpu") == (12.5, 1000.0)
    assert bench.job_value(1000, 4, 2.0) == pytest.approx(1000 * 2 * 4 / 2e-3)


def test_reference_arm_other_ranks_do_no_work(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(workload="c4", instances=2, warmup=3, steps=1)
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
