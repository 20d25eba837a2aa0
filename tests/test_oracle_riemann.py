"""Pins for the oracle's standard fluxes (MUSCL-Hancock + HLLC + van Leer,
Sec. II.C.5 last paragraph) and the moving-wall state (eq. riemann_wallvel):
closed-form Riemann properties, the paper's printed shock states, an exact
Riemann solution and directional symmetry."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs
from exact_riemann import sample, star

G = 1.4
HERE = os.path.dirname(os.path.abspath(__file__))


def cons(r, u, v, p):
    return np.array([r, r * u, r * v, p / (G - 1) + 0.5 * r * (u * u + v * v)])


def flux(q, d=0):
    r, u, v = q[0], q[1] / q[0], q[2] / q[0]
    p = (G - 1) * (q[3] - 0.5 * r * (u * u + v * v))
    un = u if d == 0 else v
    return np.array([r * un, q[1] * un + (p if d == 0 else 0), q[2] * un + (p if d == 1 else 0), un * (q[3] + p)])


def golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_states.txt")):
        if line.strip() and not line.startswith("#"):
            k, r, u, p = line.split()
            out[k] = (float(r), float(u), float(p))
    return out


def test_hllc_consistency():
    q = cons(1.3, 0.4, -0.2, 2.1)
    for d in (0, 1):
        assert np.allclose(oracle.hllc(G, d, q, q), flux(q, d), rtol=0, atol=1e-14)


def test_hllc_resolves_stationary_contact():
    qL, qR = cons(1.0, 0.0, 0.3, 1.0), cons(0.125, 0.0, -0.7, 1.0)
    F = oracle.hllc(G, 0, qL, qR)
    assert np.allclose(F, [0.0, 1.0, 0.0, 0.0], atol=1e-15)


def test_hllc_upwinds_supersonic_flow():
    qL, qR = cons(1.0, 2.5, 0.1, 1.0), cons(0.8, 2.9, -0.2, 0.7)
    assert np.array_equal(oracle.hllc(G, 0, qL, qR), flux(qL))
    assert np.array_equal(oracle.hllc(G, 0, cons(1.0, -2.5, 0, 1.0), cons(0.8, -2.9, 0, 0.7)),
                          flux(cons(0.8, -2.9, 0, 0.7)))


def test_paper_shock_states_follow_rankine_hugoniot():
    """Sec. III.B prints the Mach 1.34 stationary-shock states; the shock
    relations used to build the workloads' initial states reproduce their
    density and pressure ratios to the printed precision."""
    g = golden()
    (rL, uL, pL), (rR, uR, pR) = g["shock134_left"], g["shock134_right"]
    r2, u2, p2 = inputs.post_shock(1.34)
    assert abs(r2 - rR / rL) / r2 < 5e-3
    assert abs(p2 - pR / pL) / p2 < 5e-3
    # mass flux through the stationary shock is continuous
    assert abs(rL * uL - rR * uR) / (rL * uL) < 2e-3


def _sod_run(N, d=0, t_end=0.2):
    """1-D Sod problem as a grid invariant in the other direction."""
    nx, ny = (N, 4) if d == 0 else (4, N)
    prob = inputs.Problem("sod", nx, ny, 0.0, 0.0, 1.0 if d == 0 else 4.0 / N, 4.0 / N if d == 0 else 1.0,
                          bc=(0, 0, 2, 2) if d == 0 else (2, 2, 0, 0), cfl=0.8)
    X, Y = prob.cell_centres()
    s = X if d == 0 else Y
    left = s < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    prob.Q0 = inputs.conserved(rho, 0.0, 0.0, p)
    o = oracle.Oracle(prob)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.cfl_dt(), t_end - t)
        o.step(dt)
        t += dt
    Q = o.state()
    return (Q[0, 1, :] if d == 0 else Q[0, :, 1]), (Q if d == 0 else Q), o


def test_muscl_hancock_converges_to_exact_sod():
    errs = []
    for N in (100, 200, 400):
        rho, _, _ = _sod_run(N)
        xc = (np.arange(N) + 0.5) / N
        ex = np.array([sample(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, (x - 0.5) / 0.2)[0] for x in xc])
        errs.append(np.mean(np.abs(rho - ex)))
    assert errs[0] < 0.02
    assert errs[0] / errs[1] > 1.5 and errs[1] / errs[2] > 1.5


def test_x_and_y_sweeps_agree_on_transposed_data():
    rx, Qx, _ = _sod_run(64, d=0, t_end=0.1)
    ry, Qy, _ = _sod_run(64, d=1, t_end=0.1)
    assert np.array_equal(rx, ry)
    assert np.array_equal(Qx[1, 1, :], Qy[2, :, 1])


@pytest.mark.parametrize("un,wn", [(0.3, 0.3), (-0.2, -0.2), (0.0, 0.5), (0.4, -0.1), (-0.6, 0.2)])
def test_wall_state(un, wn):
    """Moving-wall Riemann problem (eq. riemann_wallvel): u*.n = w.n always;
    a wall moving with the fluid leaves rho and p unchanged; otherwise p* is
    the exact star pressure of the reflected Riemann problem (independent
    Newton solution) and rho* follows the shock / isentropic relation."""
    n = np.array([0.6, 0.8])
    t = np.array([-0.8, 0.6])
    u = un * n + 0.37 * t
    w = wn * n + 1.3 * t
    q = cons(1.1, u[0], u[1], 0.9)
    rs, ps, usx, usy = oracle.wall_state(G, q, n, w)
    assert abs(usx * n[0] + usy * n[1] - wn) < 1e-15
    assert abs((usx * t[0] + usy * t[1]) - 0.37) < 1e-15      # tangential velocity kept
    if un == wn:
        assert abs(rs - 1.1) < 1e-15 and abs(ps - 0.9) < 1e-15
    else:
        pex, uex = star(1.1, un, 0.9, 1.1, 2 * wn - un, 0.9)
        assert abs(uex - wn) < 1e-12
        assert abs(ps - pex) / pex < 1e-10
        rex = sample(1.1, un, 0.9, 1.1, 2 * wn - un, 0.9, wn - 1e-9)[0]
        assert abs(rs - rex) / rex < 1e-6
        assert (ps > 0.9) == (un > wn)
