"""The allocation-free classification entry point, mb_cut_cells_noalloc.

It serves callers that may not allocate device memory (an application that
forbids cudaMalloc in its real-time loop, or a plugin whose host framework
owns every device buffer): the caller passes the output arrays and the call
uses a fixed scratch array inside the library.  On two calls in a row its
volume fractions must equal those of the library's allocating path bit for
bit and the oracle's to round-off, and its class bytes must equal the classes
the oracle's geometry fixes.  Kept in a file collected last, so that a run
stopping at the first failure has run everything else first."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

pytestmark = pytest.mark.gpu

SOLID, CUT, TOUCH, MOVT = 1, 2, 8, 16


def _allocating_alpha(mb, prob, t):
    sim = mb.Sim(prob, mb.FP64)
    sim.write_state(0, prob.Q0, t)
    out = sim.read_state(0, alpha=True)
    sim.close()
    return out["alpha"]


def _oracle_classes(prob, X, Y, theta):
    """Volume fractions and the class bytes they imply, from the oracle's
    geometry at the pose (every polygon of these bodies moves, so a touched
    cell is touched by a moving polygon)."""
    a, touched, _, _ = oracle.Oracle(prob).geometry(X, Y, theta)
    t = touched.astype(bool)
    cls = np.where(a == 0.0, SOLID, 0) | np.where(t & (a > 0.0), CUT, 0) | np.where(t, TOUCH | MOVT, 0)
    return a, cls.astype(np.uint8)


def _pose(prob, t):
    X, Y = prob.U[0] * t, prob.U[1] * t
    theta = prob.a0 + prob.a1 * math.sin(prob.omega * t) if (prob.a0 or prob.a1) else 0.0
    return X, Y, theta


@pytest.mark.parametrize("case", ["cylinder", "triangle", "naca"])
def test_noalloc_matches_allocating_path_and_oracle_twice(case):
    import torch
    from paper_1711_11361_gb300 import mb
    prob = inputs.c3_naca(128) if case == "naca" else inputs.small_case(case, 96, 2.0)
    t = 0.0371
    X, Y, theta = _pose(prob, t)
    ref_alpha = _allocating_alpha(mb, prob, t)
    orc_alpha, orc_cls = _oracle_classes(prob, X, Y, theta)
    # the caller owns the outputs (allocated here by torch, not by the library)
    alpha = torch.full((prob.ny, prob.nx), -1.0, dtype=torch.float64, device="cuda")
    cls = torch.zeros((prob.ny, prob.nx), dtype=torch.uint8, device="cuda")
    for call in range(2):
        alpha.fill_(-1.0)
        cls.fill_(255)
        mb.cut_cells_noalloc(prob, X, Y, theta, alpha.data_ptr(), cls.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        a = alpha.cpu().numpy()
        c = cls.cpu().numpy()
        assert np.array_equal(a, ref_alpha), (case, call, np.max(np.abs(a - ref_alpha)))
        assert np.max(np.abs(a - orc_alpha)) <= 1e-12, (case, call)
        assert np.array_equal(c, orc_cls), (case, call, int(np.sum(c != orc_cls)))


def test_noalloc_reports_edge_capacity_then_recovers():
    """A body sampled far more finely than the grid (over 192 edges in one
    grid column) is refused with MB_E_CAPACITY instead of truncated lists;
    the next valid call on the same scratch array is exact again."""
    import torch
    from paper_1711_11361_gb300 import mb
    th = np.linspace(0.0, 2.0 * np.pi, 3000, endpoint=False)
    dense = np.stack([0.5 + 0.3 * np.cos(th), 0.5 + 0.3 * np.sin(th)], axis=1)
    prob = inputs.Problem("dense", 8, 8, 0.0, 0.0, 1.0, 1.0, polygons=[dense], moving=[1])
    a = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    c = torch.zeros((8, 8), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        with pytest.raises(mb.MBError) as ei:
            mb.cut_cells_noalloc(prob, 0.0, 0.0, 0.0, a.data_ptr(), c.data_ptr())
        assert ei.value.code == mb.MB_E_CAPACITY
    ok = inputs.small_case("cylinder", 64, 2.0)
    a2 = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    c2 = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    mb.cut_cells_noalloc(ok, 0.0, 0.0, 0.0, a2.data_ptr(), c2.data_ptr())
    torch.cuda.synchronize()
    orc_alpha, orc_cls = _oracle_classes(ok, 0.0, 0.0, 0.0)
    assert np.max(np.abs(a2.cpu().numpy() - orc_alpha)) <= 1e-13
    assert np.array_equal(c2.cpu().numpy(), orc_cls)


def test_noalloc_rejects_oversized_requests():
    from paper_1711_11361_gb300 import mb
    import torch
    prob = inputs.small_case("cylinder", 64, 2.0)
    big = inputs.Problem("big", 9000, 16, 0.0, 0.0, 1.0, 1.0, polygons=prob.polygons, moving=[1])
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    c = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(mb.MBError):
        mb.cut_cells_noalloc(big, 0.0, 0.0, 0.0, a.data_ptr(), c.data_ptr())
