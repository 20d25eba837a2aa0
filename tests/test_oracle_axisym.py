"""The geometric source of the axisymmetric Euler equations (the form the
paper's open-ended tube uses, Sec. III.E), pinned by an exact solution: a
homologous cylindrical expansion with uniform density, radial velocity
v = v0 r / (1 + v0 t), density rho0 / (1 + v0 t)^2 and isentropic pressure
solves the axisymmetric equations exactly (the pressure stays uniform, so
nothing accelerates the gas).  The planar sweeps alone give only half of the
density's decay; the source step supplies the other half."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

G = 1.4
V0 = 0.5


def expansion(ny, axisym=True, t_end=0.1):
    p = inputs.Problem("expansion", 4, ny, 0.0, 0.0, 4.0 / ny, 1.0,
                       bc=(inputs.PERIODIC, inputs.PERIODIC, inputs.REFLECTIVE, inputs.TRANSMISSIVE), cfl=0.4,
                       axisym=axisym)
    X, Y = p.cell_centres()
    p.Q0 = inputs.conserved(np.ones_like(X), 0.0, V0 * Y, np.full_like(X, 1.0 / G))
    o = oracle.Oracle(p)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(o.cfl_dt(), t_end - t)
        assert o.step(dt)[0] == 0
        t += dt
    Q = o.state()
    r = Y[:, 0]
    inner = r < 0.5                      # the outflow side's disturbance has not arrived
    rho_ex = 1.0 / (1.0 + V0 * t) ** 2
    p_ex = (1.0 / G) * rho_ex ** G
    rho = Q[0][inner, 0]
    q = Q[:, inner, 0]
    pr = (G - 1.0) * (q[3] - 0.5 * (q[1] ** 2 + q[2] ** 2) / q[0])
    v_ex = V0 * r[inner] / (1.0 + V0 * t)
    return (np.max(np.abs(rho - rho_ex)) / rho_ex, np.max(np.abs(pr - p_ex)) / p_ex,
            np.max(np.abs(q[2] / q[0] - v_ex)))


def test_expansion_matches_exact_solution_and_converges():
    e1 = expansion(32)
    e2 = expansion(64)
    assert e1[0] < 2e-3 and e1[1] < 3e-3 and e1[2] < 2e-3
    for a, b in zip(e1, e2):
        assert math.log2(a / b) > 0.8, (e1, e2)


def test_planar_sweeps_alone_miss_the_source():
    assert expansion(32, axisym=False)[0] > 1e-2


def test_source_leaves_states_without_radial_velocity_alone():
    p = inputs.Problem("axial", 8, 8, 0.0, 0.0, 1.0, 1.0, bc=(inputs.PERIODIC, inputs.PERIODIC,
                       inputs.REFLECTIVE, inputs.TRANSMISSIVE), cfl=0.5, axisym=True)
    X, Y = p.cell_centres()
    p.Q0 = inputs.conserved(np.ones_like(X), 0.7, 0.0, np.full_like(X, 1.0))
    o = oracle.Oracle(p)
    for _ in range(5):
        assert o.step()[0] == 0
    assert np.allclose(o.state(), p.Q0, rtol=0, atol=1e-14)
