"""The allocation-free classification entry point (for callers that may not
allocate device memory) matches the classification the library computes
with its own allocations, on two calls in a row.  Kept in a file collected
last so that a run stopping at the first failure has run everything else."""
import math

import numpy as np
import pytest

from paper_1711_11361_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference(mb, prob, t):
    sim = mb.Sim(prob, mb.FP64)
    sim.write_state(0, prob.Q0, t)
    out = sim.read_state(0, alpha=True)
    return out["alpha"], out


@pytest.mark.parametrize("case", ["cylinder", "triangle", "naca"])
def test_noalloc_matches_allocating_path_twice(case):
    import torch
    from paper_1711_11361_gb300 import mb
    if case == "naca":
        prob = inputs.c3_naca(128)
    else:
        prob = inputs.small_case(case, 96, 2.0)
    t = 0.0371
    ref_alpha, _ = _reference(mb, prob, t)
    X, Y = prob.U[0] * t, prob.U[1] * t
    theta = prob.a0 + prob.a1 * math.sin(prob.omega * t) if (prob.a0 or prob.a1) else 0.0
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
        assert np.max(np.abs(a - ref_alpha)) <= 1e-13, (case, call)
        assert np.array_equal((c & 1) == 1, ref_alpha == 0.0), (case, call)


def test_noalloc_rejects_oversized_requests():
    from paper_1711_11361_gb300 import mb
    import torch
    prob = inputs.small_case("cylinder", 64, 2.0)
    big = inputs.Problem("big", 9000, 16, 0.0, 0.0, 1.0, 1.0, polygons=prob.polygons, moving=[1])
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    c = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(mb.MBError):
        mb.cut_cells_noalloc(big, 0.0, 0.0, 0.0, a.data_ptr(), c.data_ptr())
