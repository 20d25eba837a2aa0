"""The sloped-channel validation case (Sec. III.A) as read in
inputs.n1_channel, on the oracle: the density pulse is carried along the
30-degree channel to its exact translated profile, with errors that fall
with the grid like the paper's static table (global L1 order above one),
for a static channel and for the moving one."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs


def l1_error(level, moving, mode=inputs.UNCOVER_DONOR):
    p = inputs.n1_channel(level, moving)
    p.uncover_mode = mode
    o = oracle.Oracle(p)
    t = 0.0
    m0 = o.contents()[0].sum()
    while t < p.t_end - 1e-14:
        dt = min(o.cfl_dt(), p.t_end - t)
        assert o.step(dt)[0] == 0
        t += dt
    X, Y = p.cell_centres()
    a, rho = o.alpha(), o.state()[0]
    fl = a > 0
    e = np.abs(rho[fl] - inputs.n1_exact_density(X, Y, t, p.U[0])[fl])
    return float(np.sum(a[fl] * e) / np.sum(a[fl])), o


def test_n1_geometry():
    p = inputs.n1_channel(0)
    a, touched, _, _ = oracle.Oracle(p).geometry()
    # channel area inside the 5 x 1 box: width 0.25 x length 1 / sin 30 = 0.5
    assert abs(a.sum() * p.dx * p.dy - 0.5) < 1e-12
    assert touched.sum() > 100


def test_n1_initial_state_is_the_exact_profile():
    p = inputs.n1_channel(0)
    X, Y = p.cell_centres()
    assert np.allclose(p.Q0[0], inputs.n1_exact_density(X, Y, 0.0, p.U[0]))


@pytest.mark.parametrize("moving,mode", [(False, inputs.UNCOVER_DONOR), (True, inputs.UNCOVER_FLUX_GCL)])
def test_n1_converges(moving, mode):
    e0, _ = l1_error(0, moving, mode)
    e1, _ = l1_error(1, moving, mode)
    assert e0 < 1e-2
    assert math.log2(e0 / e1) > 1.0
