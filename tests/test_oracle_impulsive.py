"""Why an impulsive start drives the cells in front of an advancing wall
negative (Sec. II.C.4 with the moving-wall boundary state of eq.
riemann_wallvel).

A y-invariant wall advances in +x at speed w into gas at rest.  Its cut cell
(wall inside, fluid to the right, the left face inside the body) shields its
right face completely, so that face carries F2D = FB + d (F - FB) (eqs.
Klein2DtotalfluxaMethod2, Klein2shieldedFluxMethod2) with d the cell's
volume fraction at the mid pose, while the wall term FB - w QB has no mass
(eq. Klein2DMovingResultantFluxes).  With F's mass flux 0 (gas at rest) the
cell's new mass content after the first x sweep is

    alpha_B rho' = alpha_A rho - (dt/dx) w rho* (1 - d),

where rho* > rho is the wall state's density (the paper: an advancing wall
has rho* > rho).  The cell gives away the mass flux of the compressed wall
state while it holds uncompressed gas, so once alpha_A rho < (dt/dx) w rho*
(1 - d) -- a cell in front of the wall that is nearly covered this step --
its mass turns negative.  The same cell holding gas at the wall state, or
gas moving with the wall, stays positive.  These tests check the formula on
the oracle and the sign change it predicts."""
import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

G = 1.4
NX, NY = 20, 4
DX = 1.0 / NX


def wall_problem(xw, w, rho, u, p):
    body = inputs.rect_polygon(-1.0, -1.0, xw, 2.0)
    prob = inputs.Problem("wall", NX, NY, 0.0, 0.0, 1.0, 1.0, bc=(0, 0, 0, 0), cfl=0.5, polygons=[body],
                          moving=[1], U=(w, 0.0))
    X, Y = prob.cell_centres()
    prob.Q0 = inputs.conserved(np.full_like(X, rho), u, 0.0, p)
    return prob


def first_sweep(alpha_a, lam_w, rho=1.0, u=0.0, p=1.0):
    """Cut cell 5 with volume fraction alpha_a at the start; the wall moves by
    lam_w cells in the first x sweep.  Returns (mass content of the cell after
    the sweep, predicted content, cells merged by the safeguard)."""
    c = np.sqrt(G * 1.0 / 1.0)
    w = 0.5 * c
    xw = (6 - alpha_a) * DX                 # cut cell i = 5: [0.25, 0.30]
    dt = lam_w * DX / w
    o = oracle.Oracle(wall_problem(xw, w, rho, u, p))
    a0 = o.alpha()
    assert abs(a0[1, 5] - alpha_a) < 1e-12 and a0[1, 4] == 0.0 and a0[1, 6] == 1.0
    q = np.array([rho, rho * u, 0.0, p / (G - 1.0) + 0.5 * rho * u * u])
    rs, _, _, _ = oracle.wall_state(G, q, (-1.0, 0.0), (w, 0.0))   # normal into the body: -x
    d = alpha_a - 0.5 * lam_w                 # volume fraction at the mid pose
    predicted = alpha_a * rho - lam_w * rs * (1.0 - d)
    r = o.sweep(0, dt)
    _, mixed = o.last_sweep()
    return o.contents()[0, 1, 5], predicted, mixed, r, rs


def test_wall_state_is_compressed():
    _, _, _, _, rs = first_sweep(0.5, 0.2)
    assert rs > 1.5          # the advancing wall compresses the gas at rest


@pytest.mark.parametrize("alpha_a", [0.9, 0.6, 0.45])
def test_front_cell_mass_follows_the_formula(alpha_a):
    """Cells that keep positive mass: the oracle's content equals the formula."""
    got, pred, mixed, r, _ = first_sweep(alpha_a, 0.2)
    assert r == 0 and mixed == 0
    assert pred > 0.0
    assert abs(got - pred) < 1e-12, (got, pred)


def test_nearly_covered_front_cell_turns_negative():
    """alpha_A = 0.22, wall moves 0.2 cells: alpha_B = 0.02 and the formula's
    content is negative; the oracle's positivity safeguard has to merge it."""
    _, pred, mixed, _, _ = first_sweep(0.22, 0.2)
    assert pred < 0.0
    assert mixed > 0


def test_same_cell_positive_when_it_holds_the_wall_state():
    """Started from gas already at the wall state (the post-shock density
    moving with the wall, as the piston instances start), the same nearly
    covered cell keeps its mass: alpha_A rho* - lam w rho* (1 - d) =
    rho* (alpha_B + lam w d) > 0."""
    c = np.sqrt(G)
    w = 0.5 * c
    q0 = np.array([1.0, 0.0, 0.0, 1.0 / (G - 1.0)])
    rs, ps, _, _ = oracle.wall_state(G, q0, (-1.0, 0.0), (w, 0.0))
    got, _, mixed, r, rs2 = first_sweep(0.22, 0.2, rho=rs, u=w, p=ps)
    assert abs(rs2 - rs) < 1e-9 * rs        # gas moving with the wall is not compressed further
    assert r == 0 and mixed == 0
    assert got > 0.0
