"""Pins for the oracle's cut-cell geometry (Sec. II.A volume fractions,
Sec. II.B apertures, Sec. II.C.4 swept apertures): brute-force sampling on
tiny grids, the shoelace area, the divergence-theorem closure and the exact
swept-strip geometric conservation identity."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _inside(poly, X, Y):
    """Even-odd test of points (X, Y) against polygon (vectorised brute force)."""
    x, y = poly[:, 0], poly[:, 1]
    inside = np.zeros(X.shape, dtype=bool)
    n = len(poly)
    for k in range(n):
        xa, ya, xb, yb = x[k], y[k], x[(k + 1) % n], y[(k + 1) % n]
        cross = (ya > Y) != (yb > Y)
        with np.errstate(divide="ignore", invalid="ignore"):
            xi = xa + (Y - ya) * (xb - xa) / (yb - ya)
        inside ^= cross & (X < xi)
    return inside


def _prob(polys, N, lo=0.0, hi=1.0):
    p = inputs.Problem("geom", N, N, lo, lo, hi, hi, polygons=polys, moving=[1] * len(polys))
    p.Q0 = None
    return p


def _bruteforce_alpha(poly, prob, s):
    a = np.zeros((prob.ny, prob.nx))
    off = (np.arange(s) + 0.5) / s
    for j in range(prob.ny):
        for i in range(prob.nx):
            X, Y = np.meshgrid(prob.x0 + (i + off) * prob.dx, prob.y0 + (j + off) * prob.dy)
            a[j, i] = 1.0 - _inside(poly, X, Y).mean()
    return a


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_alpha_matches_bruteforce_triangle(seed):
    rng = np.random.default_rng(seed)
    tri = inputs.triangle_polygon(0.5 + rng.uniform(-0.1, 0.1), 0.5 + rng.uniform(-0.1, 0.1), 0.55)
    prob = _prob([tri], 12)
    a, touched, _, _ = oracle.Oracle(prob).geometry()
    s = 200
    ref = _bruteforce_alpha(tri, prob, s)
    assert np.max(np.abs(a - ref)) <= 4.0 / s
    # untouched cells are exactly solid or exactly fluid
    assert set(np.unique(a[touched == 0])).issubset({0.0, 1.0})


def test_alpha_matches_bruteforce_polygon_circle():
    poly = inputs.cylinder_polygon(0.47, 0.52, 0.31, 0.125)   # 32 vertices
    prob = _prob([poly], 8)
    a, _, _, _ = oracle.Oracle(prob).geometry()
    s = 160
    ref = _bruteforce_alpha(poly, prob, s)
    assert np.max(np.abs(a - ref)) <= 4.0 / s


def _shoelace(p):
    x, y = p[:, 0], p[:, 1]
    return 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)


@pytest.mark.parametrize("body", ["cylinder", "triangle", "naca"])
def test_total_solid_area_equals_shoelace(body):
    N = 64
    if body == "cylinder":
        poly = inputs.cylinder_polygon(0.4123, 0.5377, 0.2, 1.0 / N)
    elif body == "triangle":
        poly = inputs.triangle_polygon(0.4123, 0.5377, 0.4)
    else:
        poly = inputs.naca00xx_polygon(chord=0.7, n_side=65, le=(0.1123, 0.5077))
    prob = _prob([poly], N)
    a, _, _, _ = oracle.Oracle(prob).geometry()
    solid = np.sum(1.0 - a) * prob.dx * prob.dy
    assert abs(solid - _shoelace(poly)) <= 1e-13


def test_apertures_match_line_sampling():
    tri = inputs.triangle_polygon(0.503, 0.488, 0.6)
    prob = _prob([tri], 10)
    _, _, bx, by = oracle.Oracle(prob).geometry()
    s = 20000
    t = (np.arange(s) + 0.5) / s
    for j in range(prob.ny):
        for i in range(prob.nx + 1):
            X = np.full(s, prob.x0 + i * prob.dx)
            Y = prob.y0 + (j + t) * prob.dy
            assert abs(bx[j, i] - (1.0 - _inside(tri, X, Y).mean())) <= 2.0 / s
    for j in range(prob.ny + 1):
        for i in range(prob.nx):
            Y = np.full(s, prob.y0 + j * prob.dy)
            X = prob.x0 + (i + t) * prob.dx
            assert abs(by[j, i] - (1.0 - _inside(tri, X, Y).mean())) <= 2.0 / s


def test_aperture_closure_gives_wall_length():
    """Divergence theorem on the fluid part of a cell cut by one straight edge:
    |((bW - bE) dy, (bS - bN) dx)| equals the edge length inside the cell."""
    # one large triangle; check cells cut by a single edge and no vertex
    tri = np.array([[0.1037, 0.1213], [0.9071, 0.2379], [0.4513, 0.8893]])
    N = 16
    prob = _prob([tri], N)
    a, touched, bx, by = oracle.Oracle(prob).geometry()
    checked = 0
    for j in range(N):
        for i in range(N):
            if not (0.0 < a[j, i] < 1.0):
                continue
            xl, xr, yl, yh = i / N, (i + 1) / N, j / N, (j + 1) / N
            if any(xl <= v[0] <= xr and yl <= v[1] <= yh for v in tri):
                continue
            # the single edge crossing the cell: clip each edge to the cell
            L, nedges = 0.0, 0
            for k in range(3):
                p0, p1 = tri[k], tri[(k + 1) % 3]
                t0, t1 = 0.0, 1.0
                d = p1 - p0
                for pv, qv in ((-d[0], p0[0] - xl), (d[0], xr - p0[0]), (-d[1], p0[1] - yl), (d[1], yh - p0[1])):
                    if pv == 0:
                        if qv < 0:
                            t0, t1 = 1, 0
                        continue
                    r = qv / pv
                    if pv < 0:
                        t0 = max(t0, r)
                    else:
                        t1 = min(t1, r)
                if t1 > t0:
                    L += (t1 - t0) * math.hypot(*d)
                    nedges += 1
            if nedges != 1:
                continue
            nL = math.hypot((bx[j, i] - bx[j, i + 1]) / N, (by[j, i] - by[j + 1, i]) / N)
            assert abs(nL - L) <= 1e-14
            checked += 1
    assert checked > 10


@pytest.mark.parametrize("d,delta", [(0, 0.37), (0, -0.61), (1, 0.29), (1, -0.83)])
@pytest.mark.parametrize("body", ["cylinder", "triangle"])
def test_swept_apertures_close_the_gcl_exactly(body, d, delta):
    """alpha(B) - alpha(A) = (delta/h) (beta~_lo - beta~_hi) for a translation by
    delta (a fraction of a cell) along d: the exact swept strips of
    eq. timeAveragedBeta make the discrete geometric conservation law exact."""
    N = 32
    poly = (inputs.cylinder_polygon(0.4713, 0.5209, 0.23, 1.0 / N) if body == "cylinder"
            else inputs.triangle_polygon(0.4713, 0.5209, 0.45))
    prob = _prob([poly], N)
    o = oracle.Oracle(prob)
    h = 1.0 / N
    D = delta * h
    aA, _, _, _ = o.geometry(0.0, 0.0)
    aB, _, _, _ = o.geometry(D if d == 0 else 0.0, D if d == 1 else 0.0)
    bt = o.swept(d, D)
    if d == 0:
        rhs = delta * (bt[:, :-1] - bt[:, 1:])
    else:
        rhs = delta * (bt[:-1, :] - bt[1:, :])
    assert np.max(np.abs((aB - aA) - rhs)) <= 1e-13


def test_translation_by_one_cell_shifts_fields():
    N = 24
    poly = inputs.triangle_polygon(0.4713, 0.5209, 0.45)
    o = oracle.Oracle(_prob([poly], N))
    a0, t0, bx0, by0 = o.geometry(0.0, 0.0)
    a1, t1, bx1, by1 = o.geometry(1.0 / N, 0.0)
    assert np.max(np.abs(a1[:, 1:] - a0[:, :-1])) <= 1e-12
    assert np.array_equal(t1[:, 2:-1], t0[:, 1:-2])
    assert np.max(np.abs(bx1[:, 1:] - bx0[:, :-1])) <= 1e-12


def test_touching_polygons_sum_areas():
    """Piston-in-tube bodies touch along edges; areas still add up."""
    prob = inputs.small_case("piston", 80)
    a, _, _, _ = oracle.Oracle(prob).geometry()
    solid = np.sum(1.0 - a) * prob.dx * prob.dy
    box = lambda p: max(0.0, min(p[:, 0].max(), 1.0) - max(p[:, 0].min(), 0.0)) * (p[:, 1].max() - p[:, 1].min())
    assert abs(solid - sum(box(p) for p in prob.polygons)) <= 1e-13
