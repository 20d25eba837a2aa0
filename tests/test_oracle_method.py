"""Pins for the oracle's moving-boundary sweep as a whole: discrete
conservation (Sec. II.A, II.C.5), the consistency condition of a body moving
with the fluid (Sec. II.C.1), the 1-D reduction of the stabilised cut-cell
update (Sec. II.B, eq. Klein2shieldedFlux), small-cell stability at the
regular-cell time step (abstract, Sec. II.B), the static limit (Sec. II.C.4,
last paragraph) and the paper's printed piston-driven shock (Sec. III.E)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

G = 1.4
HERE = os.path.dirname(os.path.abspath(__file__))
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def periodic_body_problem(kind, N, U, mode, state="uniform", M=2.0):
    dx = 1.0 / N
    if kind == "cylinder":
        polys = [inputs.cylinder_polygon(0.4713, 0.5209, 0.17, dx)]
    elif kind == "triangle":
        polys = [inputs.triangle_polygon(0.4713, 0.5209, 0.3)]
    else:
        polys = [inputs.naca00xx_polygon(chord=0.5, n_side=33, le=(0.2313, 0.5209))]
    prob = inputs.Problem(f"periodic_{kind}", N, N, 0.0, 0.0, 1.0, 1.0, bc=(2, 2, 2, 2), cfl=0.5,
                          polygons=polys, moving=[1], U=U, pivot=(0.4713, 0.5209), uncover_mode=mode)
    X, Y = prob.cell_centres()
    if state == "uniform":
        prob.Q0 = inputs.conserved(np.ones_like(X), U[0], U[1], 1.0)
    else:
        rho = 1.0 + 0.3 * np.exp(-((X - 0.8) ** 2 + (Y - 0.3) ** 2) / 0.01)
        p = 1.0 + 0.5 * np.exp(-((X - 0.2) ** 2 + (Y - 0.7) ** 2) / 0.02)
        prob.Q0 = inputs.conserved(rho, 0.3 + 0.2 * np.sin(2 * np.pi * Y), -0.1 + 0.1 * np.cos(2 * np.pi * X), p)
    return prob


def total(o):
    return o.contents().sum(axis=(1, 2))


@pytest.mark.parametrize("kind", ["cylinder", "triangle", "naca"])
def test_static_body_conserves_mass_and_energy(kind):
    """Static walls: the common advective wall state of both sweeps and the
    closure normal make the wall's mass and energy terms cancel per step."""
    o = oracle.Oracle(periodic_body_problem(kind, 48, (0.0, 0.0), 0, state="bumpy"))
    m0 = total(o)
    for _ in range(30):
        r, _ = o.step()
        assert r == 0
    m1 = total(o)
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-13
    assert abs(m1[3] - m0[3]) / m0[3] < 1e-13


@pytest.mark.parametrize("mode", [inputs.UNCOVER_DONOR, inputs.UNCOVER_FLUX_GCL])
@pytest.mark.parametrize("kind,U", [("cylinder", (0.45, 0.2)), ("triangle", (-0.3, 0.55)), ("naca", (0.6, -0.15))])
def test_contents_change_only_by_wall_terms(kind, U, mode):
    """Per sweep, sum(alpha Q) changes by exactly the sum of the wall terms:
    face fluxes telescope and covering, uncovering and the positivity
    safeguard only move content between cells."""
    o = oracle.Oracle(periodic_body_problem(kind, 40, U, mode, state="bumpy"))
    dt = o.cfl_dt()
    scale = np.abs(total(o)).max()
    for k in range(24):
        for d in ((0, 1) if k % 2 == 0 else (1, 0)):
            c0 = total(o)
            assert o.sweep(d, dt) == 0
            wall, _ = o.last_sweep()
            assert np.max(np.abs(total(o) - c0 - wall)) / scale < 1e-13


@pytest.mark.parametrize("kind,U", [("cylinder", (0.45, 0.2)), ("triangle", (-0.3, 0.55)), ("naca", (0.6, -0.15))])
def test_uniform_flow_with_comoving_body_stays_uniform(kind, U):
    """Consistency condition (Sec. II.C.1, Sec. III.B): a body translating with
    a uniform flow produces no waves.  Exact with swept apertures and the
    flux-GCL treatment of uncovered cells."""
    o = oracle.Oracle(periodic_body_problem(kind, 40, U, inputs.UNCOVER_FLUX_GCL))
    ref = inputs.conserved(1.0, U[0], U[1], 1.0)
    for _ in range(60):
        assert o.step()[0] == 0
    # 60 steps keep the body inside the box (bodies do not wrap across
    # periodic sides).  The scheme is exact for this flow; what remains is
    # round-off amplified by 1/alpha in the smallest cut cells (~2e-9 seen);
    # an O(dx) inconsistency would show up at 1e-3 or more.
    Q, a = o.state(), o.alpha()
    dev = max(np.nanmax(a * np.abs(Q[c] - ref[c])) for c in range(4)) / np.abs(ref).max()
    assert dev < 1e-8
    big = a > 0.01
    assert max(np.max(np.abs(Q[c][big] - ref[c])) for c in range(4)) / np.abs(ref).max() < 1e-8


def test_uniform_flow_donor_mode_deviation_is_bounded():
    """Paper-literal uncovering (eqs. volumeWeighting .. DonorCellUpdate)
    lowers the donors' state by the fraction they give away (Sec. II.C.5
    names this penalty); the flow is no longer exactly uniform but stays
    close to it, while contents remain exactly conserved (tested above)."""
    U = (0.45, 0.2)
    o = oracle.Oracle(periodic_body_problem("cylinder", 40, U, inputs.UNCOVER_DONOR))
    for _ in range(30):
        assert o.step()[0] == 0
    rel = np.abs(o.state()[0] - 1.0)
    assert 1e-6 < np.nanmax(rel) < 0.5


def wall_problem(alpha, N=32, cfl=0.8, rho_u=0.0, ny=4):
    """1-D channel with a static vertical wall inside cell k = N//2 such that
    that cell's fluid fraction is alpha (fluid on the left)."""
    dx = 1.0 / N
    k = N // 2
    xw = k * dx + alpha * dx
    body = np.array([[xw, -1.0], [1.5, -1.0], [1.5, 2.0], [xw, 2.0]])
    prob = inputs.Problem("wall1d", N, ny, 0.0, 0.0, 1.0, ny * dx, bc=(1, 1, 2, 2), cfl=cfl,
                          polygons=[body], moving=[0])
    return prob, k


def test_one_dimensional_reduction_removes_alpha():
    """With the wall in cell k and uniform data moving toward it, the cut
    cell's update is Q + (dt/dx)(F(Q) - F^B) for every alpha: the stabilised
    shielded flux cancels the 1/alpha of the plain cut-cell update
    (eqs. Klein2shieldedFlux, Klein2DalphaHat with d = alpha in 1-D)."""
    outs, alphas = [], (0.7, 0.3, 1e-3, 1e-7)
    for alpha in alphas:
        prob, k = wall_problem(alpha)
        X, _ = prob.cell_centres()
        prob.Q0 = inputs.conserved(np.ones_like(X), 0.3, 0.1, 1.0)
        o = oracle.Oracle(prob)
        dt = 0.01
        assert o.sweep(0, dt) == 0
        outs.append(o.state()[:, 1, k])
    q = inputs.conserved(1.0, 0.3, 0.1, 1.0)
    rs, ps, usx, usy = oracle.wall_state(G, q, (1.0, 0.0), (0.0, 0.0))
    F = np.array([0.3, 0.3 * 0.3 + 1.0, 0.3 * 0.1, 0.3 * (q[3] + 1.0)])
    FB = np.array([0.0, ps, 0.0, 0.0])
    ref = q + 0.01 * 32 * (F - FB)
    for alpha, out in zip(alphas, outs):
        # round-off of the contents is divided by alpha once
        assert np.max(np.abs(out - ref)) < 1e-13 + 1e-15 / alpha


@pytest.mark.parametrize("alpha", [0.1, 1e-3, 1e-6, 1e-9])
def test_small_cells_stable_at_regular_time_step(alpha):
    """Small-cell problem (abstract; Sec. II.B): a tiny cut cell stays bounded at
    CFL 0.8 on regular cells for many steps of a sloshing flow."""
    prob, k = wall_problem(alpha, N=32, cfl=0.8)
    X, _ = prob.cell_centres()
    prob.Q0 = inputs.conserved(1.0 + 0.5 * np.exp(-((X - 0.2) / 0.05) ** 2), 0.2, 0.0, 1.0)
    o = oracle.Oracle(prob)
    for _ in range(600):
        assert o.step()[0] == 0
    Q = o.state()
    assert np.nanmax(np.abs(Q)) < 10.0
    assert np.nanmin(Q[0]) > 0.2


def test_static_limit_is_continuous():
    """As the body speed goes to zero the moving scheme approaches the static
    one (Sec. II.C.4, last paragraph)."""
    res = []
    for U in (0.0, 1e-9, 1e-8):
        o = oracle.Oracle(periodic_body_problem("triangle", 32, (U, 0.5 * U), inputs.UNCOVER_DONOR, state="bumpy"))
        dt = 0.004
        for _ in range(5):
            o.step(dt)
        res.append(np.nan_to_num(o.contents()))
    d1 = np.max(np.abs(res[1] - res[0]))
    d2 = np.max(np.abs(res[2] - res[0]))
    assert 0 < d1 < 1e-7
    assert 3 < d2 / d1 < 30        # first order in the body speed


def golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_states.txt")):
        if line.strip() and not line.startswith("#"):
            k, r, u, p = line.split()
            out[k] = (float(r), float(u), float(p))
    return out


def test_piston_plateau_matches_paper_state():
    """Sec. III.E: a piston moving at 337.974 m/s into air at rest
    (1.225 kg/m^3, 101325 Pa) drives a Mach 1.76 shock with 2.812 kg/m^3 and
    349288 Pa behind it.  A planar piston run of the full method (moving cut
    cells, covering) reproduces the printed plateau."""
    g = golden()
    r1, _, p1 = g["piston176_ahead"]
    r2, up, p2 = g["piston176_behind"]
    c1 = math.sqrt(G * p1 / r1)
    N, ny = 240, 4
    dx = 1.0 / N
    xf = 0.1 + 0.3713 * dx
    body = np.array([[-0.3, -1.0], [xf, -1.0], [xf, 2.0], [-0.3, 2.0]])
    prob = inputs.Problem("piston1d", N, ny, 0.0, 0.0, 1.0, ny * dx, bc=(0, 0, 2, 2), cfl=0.5,
                          polygons=[body], moving=[1], U=(up / c1, 0.0))
    X, _ = prob.cell_centres()
    prob.Q0 = inputs.conserved(np.ones_like(X), 0.0, 0.0, 1.0 / G)
    o = oracle.Oracle(prob)
    t = 0.0
    while t < 0.3:
        r, dt = o.step()
        assert r == 0
        t += dt
    Q = o.state()[:, 1, :]
    xs = o.clock()["X"] + xf
    shock = xs + 0.0  # plateau lies between the piston face and the shock
    Ms = 1.76
    xshock = xf + Ms * t
    xc = (np.arange(N) + 0.5) * dx
    sel = (xc > xs + 0.05) & (xc < xshock - 0.05)
    rho = Q[0, sel]
    p = (G - 1) * (Q[3, sel] - 0.5 * Q[1, sel] ** 2 / Q[0, sel])
    assert sel.sum() > 20
    assert abs(rho.mean() - r2 / r1) / (r2 / r1) < 0.01
    assert abs(p.mean() * G - p2 / p1) / (p2 / p1) < 0.01
