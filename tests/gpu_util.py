"""Helpers shared by the GPU parity tests (comparison of the CUDA path with
the oracle on the same seeded inputs)."""
import numpy as np

import oracle


def contents(Q, alpha):
    return np.where(alpha[None] > 0, alpha[None] * np.nan_to_num(Q), 0.0)


def rel_linf(a, b):
    """Per-component max |a - b| / max |b| over contents alpha*Q.  A component
    that vanishes by symmetry (rho*v of a flow symmetric about y = const) is
    measured against 1e-2 of the largest component's scale instead of its own
    round-off-sized maximum."""
    scales = [np.max(np.abs(b[c])) for c in range(b.shape[0])]
    floor = 1e-2 * max(scales) if max(scales) > 0 else 1.0
    return max(np.max(np.abs(a[c] - b[c])) / max(scales[c], floor) for c in range(a.shape[0]))


def compare(sim, orc, inst=0):
    g = sim.read_state(inst, alpha=True)
    ag, Qg = g["alpha"], g["Q"]
    ao, Qo = orc.alpha(), orc.state()
    return dict(alpha=np.max(np.abs(ag - ao)), cls=int(np.sum((ag > 0) != (ao > 0))),
                contents=rel_linf(contents(Qg, ag), contents(Qo, ao)), g=g)
