"""Seeded synthetic problem descriptions (bodies, motions, initial states).

This module holds no arithmetic of the cut-cell method: it only lays out the
inputs both the CUDA library and the CPU oracle consume -- grid extents,
boundary conditions, body polygons at t = 0 (counter-clockwise, a union of
polygons with disjoint interiors), the rigid motion, and cell-centre initial
states in conserved variables.  The workloads are shaped like the paper's
test cases (Sec. III): a density pulse in an inclined channel, a cylinder
meeting a normal shock, a triangular wedge, a piston in a tube and a pitching
NACA 0012 aerofoil.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

EULER, ADVECTION = 0, 1
TRANSMISSIVE, REFLECTIVE, PERIODIC = 0, 1, 2
UNCOVER_DONOR, UNCOVER_FLUX_GCL = 0, 1
BASE_SEED = 1711113610
GAMMA = 1.4


@dataclass
class Problem:
    """One simulation instance."""
    name: str
    nx: int
    ny: int
    x0: float
    y0: float
    x1: float
    y1: float
    bc: tuple = (TRANSMISSIVE,) * 4          # x-low, x-high, y-low, y-high
    equation: int = EULER
    adv: tuple = (0.0, 0.0)
    gamma: float = GAMMA
    cfl: float = 0.5
    uncover_mode: int = UNCOVER_DONOR
    polygons: List[np.ndarray] = field(default_factory=list)   # each (n, 2), CCW
    moving: List[int] = field(default_factory=list)
    U: tuple = (0.0, 0.0)
    pivot: tuple = (0.0, 0.0)
    a0: float = 0.0
    a1: float = 0.0
    omega: float = 0.0
    Q0: Optional[np.ndarray] = None           # (nc, ny, nx) conserved variables
    steps: int = 0
    t_end: float = 0.0
    axisym: bool = False                      # Euler in axisymmetric form (y: radius from the axis y = y0)

    @property
    def nc(self) -> int:
        return 4 if self.equation == EULER else 1

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    def cell_centres(self):
        xc = self.x0 + (np.arange(self.nx) + 0.5) * self.dx
        yc = self.y0 + (np.arange(self.ny) + 0.5) * self.dy
        return np.meshgrid(xc, yc)


# --------------------------------------------------------------------------
# bodies (counter-clockwise vertex lists)
# --------------------------------------------------------------------------
def cylinder_polygon(cx, cy, r, dx):
    """Regular polygon inscribed in the circle, about two vertices per cell width."""
    n = 4 * max(4, math.ceil(math.pi * r / dx))
    th = 2.0 * math.pi * np.arange(n) / n
    return np.stack([cx + r * np.cos(th), cy + r * np.sin(th)], axis=1)


def triangle_polygon(cx, cy, side):
    """Equilateral triangle with centroid (cx, cy), apex pointing to +x."""
    R = side / math.sqrt(3.0)
    th = np.array([0.0, 2.0 * math.pi / 3.0, 4.0 * math.pi / 3.0])
    return np.stack([cx + R * np.cos(th), cy + R * np.sin(th)], axis=1)


def naca00xx_polygon(t=0.12, chord=1.0, n_side=257, le=(-0.25, 0.0)):
    """Symmetric NACA 4-digit section from the standard thickness formula,
    cosine-spaced; the open trailing edge is closed by a straight segment."""
    k = np.arange(n_side)
    xs = 0.5 * chord * (1.0 - np.cos(np.pi * k / (n_side - 1)))
    xi = xs / chord
    yt = 5.0 * t * chord * (0.2969 * np.sqrt(xi) - 0.1260 * xi - 0.3516 * xi ** 2
                            + 0.2843 * xi ** 3 - 0.1015 * xi ** 4)
    lower = np.stack([xs, -yt], axis=1)                 # leading edge -> trailing edge
    upper = np.stack([xs[::-1], yt[::-1]], axis=1)[:-1]  # trailing edge -> just before LE
    pts = np.concatenate([lower, upper], axis=0)
    pts[:, 0] += le[0]
    pts[:, 1] += le[1]
    return pts


def rect_polygon(xa, ya, xb, yb):
    return np.array([[xa, ya], [xb, ya], [xb, yb], [xa, yb]], dtype=np.float64)


def channel_polygons(width=0.2, xlo=-0.3, xhi=1.3):
    """Solid parts of the doubly periodic unit box around the slope-1/2 channel
    whose axis copies are -x + 2y = 0.5 + k: the strips between channel copies,
    extended past the box so that no polygon edge lies on a box side."""
    h = 0.5 * width * math.sqrt(5.0)      # half-width in units of (-x + 2y)
    polys = []
    for k in range(-3, 3):
        A = 0.5 + k + h
        B = 1.5 + k - h
        if (B + xhi) / 2.0 < -0.2 or (A + xlo) / 2.0 > 1.2:
            continue
        polys.append(np.array([[xlo, (A + xlo) / 2.0], [xhi, (A + xhi) / 2.0],
                               [xhi, (B + xhi) / 2.0], [xlo, (B + xlo) / 2.0]], dtype=np.float64))
    return polys


# --------------------------------------------------------------------------
# initial states
# --------------------------------------------------------------------------
def conserved(rho, u, v, p, gamma=GAMMA):
    rho, u, v, p = np.broadcast_arrays(*[np.asarray(a, dtype=np.float64) for a in (rho, u, v, p)])
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


def post_shock(M, rho1=1.0, p1=1.0, gamma=GAMMA):
    """Rankine-Hugoniot state behind a normal shock of Mach M running in -x
    into gas at rest: (rho2, u2, p2)."""
    c1 = math.sqrt(gamma * p1 / rho1)
    rho2 = rho1 * (gamma + 1.0) * M * M / ((gamma - 1.0) * M * M + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (M * M - 1.0))
    u2 = -2.0 / (gamma + 1.0) * (M - 1.0 / M) * c1
    return rho2, u2, p2


def shock_state(prob: Problem, M, x_shock, u_pre=0.0, gamma=GAMMA):
    """Gas at rest relative to u_pre (rho = 1, p = 1) for x < x_shock and the
    state behind a Mach-M shock running into it (toward -x) for x > x_shock."""
    X, _ = prob.cell_centres()
    r2, u2, p2 = post_shock(M, gamma=gamma)
    right = X > x_shock
    rho = np.where(right, r2, 1.0)
    u = np.where(right, u_pre + u2, u_pre)
    p = np.where(right, p2, 1.0)
    return conserved(rho, u, 0.0 * rho, p, gamma)


def piston_shock(u_p, rho1=1.0, p1=1.0, gamma=GAMMA):
    """Planar piston at speed u_p into gas at rest: shock Mach number, shock
    speed and the uniform state between piston and shock (rho2, u_p, p2)."""
    c1 = math.sqrt(gamma * p1 / rho1)
    a = (gamma + 1.0) * u_p / (4.0 * c1)
    Ms = a + math.sqrt(a * a + 1.0)
    rho2 = rho1 * (gamma + 1.0) * Ms * Ms / ((gamma - 1.0) * Ms * Ms + 2.0)
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (Ms * Ms - 1.0))
    return Ms, Ms * c1, rho2, p2


def channel_arclength(x, y):
    """Arc length along the closed slope-1/2 channel loop from (0, 0.25)."""
    L = math.sqrt(5.0)
    k = np.rint(-x + 2.0 * y - 0.5)
    s = (2.0 * (x + k) + y - 0.25) / L
    return np.mod(s, L)


def channel_pulse(s, t=0.0, s0=0.3, w=0.05):
    """Exact transported profile u0(s - t) on the loop of length sqrt(5)."""
    L = math.sqrt(5.0)
    r = np.mod(s - t - s0 + 0.5 * L, L) - 0.5 * L
    return np.exp(-(r / w) ** 2)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def c1_advection(N=100, steps=200):
    """Scalar advection along the inclined channel, doubly periodic unit box,
    CFL 0.8 on regular cells, static walls."""
    a = (2.0 / math.sqrt(5.0), 1.0 / math.sqrt(5.0))
    prob = Problem("c1_channel_advection", N, N, 0.0, 0.0, 1.0, 1.0, bc=(PERIODIC,) * 4,
                   equation=ADVECTION, adv=a, cfl=0.8, polygons=channel_polygons(),
                   moving=[0] * len(channel_polygons()), steps=steps)
    X, Y = prob.cell_centres()
    prob.Q0 = channel_pulse(channel_arclength(X, Y))[None]
    return prob


# --------------------------------------------------------------------------
# the paper's sloped-channel validation (Sec. III.A), as read here
# --------------------------------------------------------------------------
N1_ANGLE = math.radians(30.0)   # channel walls against the x-axis
N1_HALF_WIDTH = 0.125           # channel width 0.02 m in a 0.08 m high box
N1_CENTRE = (1.2, 0.5)          # point of the channel axis at mid-height (t = 0)
N1_U_AXIAL = 0.5                # gas velocity along the channel, relative to the walls
N1_AMPLITUDE, N1_WIDTH = 0.2, 0.1
N1_S0 = -0.4                    # pulse centre on the channel axis at t = 0 (from N1_CENTRE)
N1_TRAVEL = 0.8                 # distance the pulse travels along the channel by t_end


def n1_axis():
    return np.array([math.cos(N1_ANGLE), math.sin(N1_ANGLE)])


def n1_exact_density(x, y, t, V):
    """Exact density of the sloped-channel case at time t: the Gaussian
    profile along the channel axis translated with the gas velocity (a
    contact wave in a uniform flow at uniform pressure)."""
    a = n1_axis()
    ug = np.array([V + N1_U_AXIAL * a[0], N1_U_AXIAL * a[1]])
    s = (x - N1_CENTRE[0]) * a[0] + (y - N1_CENTRE[1]) * a[1] - N1_S0 - float(ug @ a) * t
    return 1.0 + N1_AMPLITUDE * np.exp(-(s / N1_WIDTH) ** 2)


def n1_channel(level=0, moving=True, cfl=0.5):
    """The paper's sloped-channel validation (Sec. III.A) as read here, in
    units of the box height (0.08 m) and the sound speed (c = 1):
    - box 5 x 1 (0.4 m x 0.08 m), grid 160x32 at level 0, doubled per level
      (the paper's 160x32 ... 2560x512);
    - two parallel walls at 30 degrees, channel width 0.25 (0.02 m); the solid
      parts are two parallelograms reaching past the box;
    - moving: the walls translate in +x at V = 0.3 (static: V = 0);
    - gas at p = 1/gamma moving with the walls plus 0.5 along the channel, so
      that it flows along the walls in their frame and their motion exerts no
      force (the paper removes that force to compare with a static channel);
    - a Gaussian density perturbation (amplitude 0.2, width 0.1) along the
      axis, uniform across the channel; exact solution: its translation with
      the gas velocity, by 0.8 along the channel at t_end;
    - transmissive box sides, CFL 0.5 (the paper's), donor-mode uncovering."""
    nx, ny = 160 * 2 ** level, 32 * 2 ** level
    V = 0.3 if moving else 0.0
    a = n1_axis()
    nrm = np.array([-a[1], a[0]])
    c = np.array(N1_CENTRE)
    L = 8.0
    polys = []
    for side in (-1.0, 1.0):
        o = c + side * N1_HALF_WIDTH * nrm
        far = o + side * 3.0 * nrm
        p0, p1 = o - L * a, o + L * a
        q1, q0 = far + L * a, far - L * a
        quad = np.array([p0, p1, q1, q0]) if side < 0 else np.array([p1, p0, q0, q1])
        # counter-clockwise
        area = 0.5 * np.sum(quad[:, 0] * np.roll(quad[:, 1], -1) - np.roll(quad[:, 0], -1) * quad[:, 1])
        polys.append(quad if area > 0 else quad[::-1].copy())
    ug = np.array([V + N1_U_AXIAL * a[0], N1_U_AXIAL * a[1]])
    t_end = N1_TRAVEL / float(ug @ a)
    prob = Problem(f"n1_channel_{'moving' if moving else 'static'}_{nx}x{ny}", nx, ny, 0.0, 0.0, 5.0, 1.0,
                   bc=(TRANSMISSIVE,) * 4, cfl=cfl, polygons=polys, moving=[1, 1], U=(V, 0.0), t_end=t_end)
    X, Y = prob.cell_centres()
    rho = n1_exact_density(X, Y, 0.0, V)
    prob.Q0 = conserved(rho, ug[0], ug[1], np.full_like(rho, 1.0 / GAMMA))
    return prob


# --------------------------------------------------------------------------
# the paper's axisymmetric open-ended tube (Sec. III.E), as read here
# --------------------------------------------------------------------------
N2_MACH = 1.76
N2_EXIT = 6.0          # tube exit plane (the tube runs from the left side)
N2_PISTON = 0.5        # piston face at t = 0 (5.5 D from the exit)
N2_WALL = 0.1          # tube wall thickness (not given in the paper; a reading)
N2_PROBE = 1.5         # pressure probe: on the axis, 1.5 D downstream of the exit


def n2_piston_speed(M=N2_MACH, gamma=GAMMA):
    """Piston speed that drives a Mach-M shock into gas at rest (rho = p = 1)."""
    c1 = math.sqrt(gamma)
    return 2.0 / (gamma + 1.0) * (M - 1.0 / M) * c1


def n2_open_tube(cells_per_d=94, t_after_exit=1.2):
    """The paper's axisymmetric open-ended tube (Sec. III.E) as read here, in
    units of the tube diameter D and the pre-shock state (rho = p = 1):
    - box 10 D x 4 D, x axial, y the radius (reflective axis at y = 0,
      transmissive elsewhere), cells_per_d cells per D (the paper's 1.6 mm,
      0.8 mm and 0.4 mm cells are about 94, 189 and 378 per D for the D that
      its shock-exit time implies, 0.151 m);
    - the tube: a fixed wall of thickness 0.1 D (not given) at radius 0.5 D
      from outside the box to the exit plane x = 6 D;
    - the piston: a rod filling the tube from outside the box to its face at
      x = 0.5 D (5.5 D from the exit), moving at the speed that drives a
      Mach 1.76 shock into gas at rest (0.993 c);
    - gas at rest, started from the exact planar piston solution at the time
      the shock is three cells ahead of the piston face (not impulsively);
    - body sides kept off the grid lines by a fraction of a cell;
    - run until t_after_exit after the planar shock reaches the exit."""
    k = cells_per_d
    if k < 25:
        # the tube wall must span a few cells: content exchanges between face
        # neighbours (covering, the safeguard) would otherwise cross it
        raise ValueError("n2_open_tube needs at least 25 cells per diameter (tube wall >= 2.5 cells)")
    nx, ny = 10 * k, 4 * k
    d = 1.0 / k
    off, ox = 0.3183 * d, 0.2718 * d
    up = n2_piston_speed()
    r_in = 0.5 + off
    tube = rect_polygon(-0.5, r_in, N2_EXIT + ox, r_in + N2_WALL)
    rod = rect_polygon(-20.0, -0.1, N2_PISTON + ox, r_in)
    Ms, S, r2, p2 = piston_shock(up)
    face = N2_PISTON + ox
    shock = face + 3.0 * d * S / (S - up)
    t_exit = (N2_EXIT + ox - shock) / S
    prob = Problem(f"n2_open_tube_{k}perD", nx, ny, 0.0, 0.0, 10.0, 4.0,
                   bc=(TRANSMISSIVE, TRANSMISSIVE, REFLECTIVE, TRANSMISSIVE), cfl=0.5, polygons=[tube, rod],
                   moving=[0, 1], U=(up, 0.0), pivot=(0.0, 0.0), axisym=True, t_end=t_exit + t_after_exit)
    X, Y = prob.cell_centres()
    inside = (X + 0.5 * d > face) & (X < shock) & (Y < r_in)
    prob.Q0 = conserved(np.where(inside, r2, 1.0), np.where(inside, up, 0.0), 0.0, np.where(inside, p2, 1.0))
    prob.n2 = dict(t_exit=t_exit, shock_speed=S, post_shock=(r2, up, p2), mach=Ms,
                   probe_cell=(int((N2_EXIT + ox + N2_PROBE) / d), 0), exit_cell=(int((N2_EXIT + ox) / d), 0))
    return prob


# a column covered from 0.3 to 0.002 of its volume in one x sweep
COLLAPSE_SLAB_DT = 0.298 / 32.0


def collapse_slab(uniform=True):
    """32^2 unit box, transmissive sides; a slab x < 19.7/32 (rows 9.32 ..
    22.32 of 32) moving at (1, 0).  In one x sweep of COLLAPSE_SLAB_DT its
    front face moves 0.298 of a cell, so the cells of column 19 the slab
    spans go from volume fraction 0.3 to 0.002.  Gas moving with the slab at
    rho = p = 1 (uniform), or a smooth non-uniform state."""
    d = 1.0 / 32.0
    slab = rect_polygon(-1.0, (9 + 0.3183) * d, 19.7 * d, (22 + 0.3183) * d)
    prob = Problem("collapse_slab", 32, 32, 0.0, 0.0, 1.0, 1.0, bc=(TRANSMISSIVE,) * 4, cfl=0.5, polygons=[slab],
                   moving=[1], U=(1.0, 0.0))
    X, Y = prob.cell_centres()
    if uniform:
        prob.Q0 = conserved(np.ones_like(X), 1.0, 0.0, np.ones_like(X))
    else:
        tp = 2.0 * math.pi
        prob.Q0 = conserved(1.0 + 0.2 * np.sin(tp * Y) + 0.1 * np.cos(tp * X), 1.0 + 0.1 * np.sin(tp * (X + Y)),
                            0.1 * np.cos(tp * X), 1.0 + 0.1 * np.sin(tp * X))
    return prob


def c2_cylinder(N=400, M=2.0, t_end=0.3, uncover_mode=UNCOVER_DONOR):
    """Cylinder r = 0.1 from (0.15, 0.5) at (0.5 c, 0) meeting a Mach-M shock at
    x = 0.3.  As in the paper's cylinder and wedge tests the body moves with
    the pre-shock gas, which is at rest in the body's frame."""
    dx = 1.0 / N
    c_inf = math.sqrt(GAMMA)
    prob = Problem("c2_cylinder_shock", N, N, 0.0, 0.0, 1.0, 1.0, cfl=0.5,
                   polygons=[cylinder_polygon(0.15, 0.5, 0.1, dx)], moving=[1],
                   U=(0.5 * c_inf, 0.0), pivot=(0.15, 0.5), t_end=t_end, uncover_mode=uncover_mode)
    prob.Q0 = shock_state(prob, M, 0.3, u_pre=0.5 * c_inf)
    return prob


def c3_naca(N=1024, periods=1.0):
    """NACA 0012, chord 1, pitching 2.5 deg sin(omega t) about the quarter chord,
    Mach 0.6 free stream (rho = 1, p = 1/gamma, c = 1), reduced frequency 0.08."""
    u_inf = 0.6
    omega = 2.0 * 0.08 * u_inf / 1.0
    prob = Problem("c3_naca0012_pitching", N, N, -2.0, -2.0, 2.0, 2.0, cfl=0.5,
                   polygons=[naca00xx_polygon()], moving=[1], pivot=(0.0, 0.0),
                   a0=0.0, a1=math.radians(2.5), omega=omega, t_end=periods * 2.0 * math.pi / omega)
    X, _ = prob.cell_centres()
    prob.Q0 = conserved(np.ones_like(X), u_inf, 0.0, 1.0 / GAMMA)
    return prob


def _body_instance(kind, N, M, uncover_mode=UNCOVER_DONOR, y_nudge=0.3183, x_nudge=0.2718):
    """One C4/C5-style instance on the unit box with a body of `kind`.
    Cylinder and triangle move with the pre-shock gas; the piston drives its
    own shock and starts from the exact planar piston solution at the time
    the shock is three cells ahead of the piston face."""
    dx = 1.0 / N
    c_inf = math.sqrt(GAMMA)
    if kind == "cylinder":
        polys, mov, U = [cylinder_polygon(0.15, 0.5, 0.1, dx)], [1], (0.5 * c_inf, 0.0)
        pivot = (0.15, 0.5)
    elif kind == "triangle":
        polys, mov, U = [triangle_polygon(0.15, 0.5, 0.2)], [1], (0.5 * c_inf, 0.0)
        pivot = (0.15, 0.5)
    elif kind == "piston":
        off, ox = y_nudge * dx, x_nudge * dx      # keep body sides off the grid lines
        polys = [rect_polygon(-0.1, 0.36 + off, 0.6 + ox, 0.40 + off),
                 rect_polygon(-0.1, 0.60 + off, 0.6 + ox, 0.64 + off),
                 rect_polygon(0.05 + ox, 0.40 + off, 0.10 + ox, 0.60 + off)]
        mov, U, pivot = [0, 0, 1], (0.3 * c_inf, 0.0), (0.075, 0.5)
    else:
        raise ValueError(kind)
    prob = Problem(f"{kind}_N{N}", N, N, 0.0, 0.0, 1.0, 1.0, cfl=0.5, polygons=polys, moving=mov,
                   U=U, pivot=pivot, uncover_mode=uncover_mode)
    if kind == "piston":
        X, Y = prob.cell_centres()
        Ms, S, r2, p2 = piston_shock(U[0])
        face = 0.10 + ox
        shock = face + 3.0 * dx * S / (S - U[0])
        inside = (X + 0.5 * dx > face) & (X < shock) & (Y > 0.40 + off) & (Y < 0.60 + off)
        prob.Q0 = conserved(np.where(inside, r2, 1.0), np.where(inside, U[0], 0.0), 0.0,
                            np.where(inside, p2, 1.0))
    else:
        prob.Q0 = shock_state(prob, M, 0.3, u_pre=U[0])
    return prob


def c4_batch(n=64, nmin=128, nmax=1024, steps=500, seed=None, kinds=("cylinder", "triangle", "piston")):
    """64 independent instances on uneven grids, seeded."""
    ss = np.random.SeedSequence(BASE_SEED).spawn(5)[3] if seed is None else np.random.SeedSequence(seed)
    rng = np.random.default_rng(ss)
    probs = []
    for k in range(n):
        N = int(rng.integers(nmin, nmax + 1))
        kind = kinds[int(rng.integers(0, len(kinds)))]
        M = float(rng.uniform(1.2, 3.0))
        p = _body_instance(kind, N, M)
        p.name = f"c4_{k:02d}_{kind}_N{N}_M{M:.3f}"
        p.steps = steps
        probs.append(p)
    return probs


def c5_requests(n=2000, nmin=256, nmax=2048, smin=500, smax=5000, seed=None,
                kinds=("cylinder", "triangle", "piston", "naca")):
    """Served stream: n request specs (kind, N, shock Mach, steps), grid size
    log-uniform in [nmin, nmax], steps uniform in [smin, smax], body uniform
    over the kinds (the pitching NACA 0012 of c3_naca; the others as in the
    batch), seeded (child 4 of the base seed).  Specs are light; make_request
    builds the problem when it is submitted."""
    ss = np.random.SeedSequence(BASE_SEED).spawn(5)[4] if seed is None else np.random.SeedSequence(seed)
    rng = np.random.default_rng(ss)
    out = []
    for k in range(n):
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        kind = kinds[int(rng.integers(0, len(kinds)))]
        M = float(rng.uniform(1.2, 3.0))
        steps = int(rng.integers(smin, smax + 1))
        out.append(dict(k=k, kind=kind, N=N, M=M, steps=steps))
    return out


def make_request(spec) -> Problem:
    """The problem of a served-stream spec (c5_requests)."""
    if spec["kind"] == "naca":
        p = c3_naca(spec["N"])
    else:
        p = _body_instance(spec["kind"], spec["N"], spec["M"])
    p.name = f"c5_{spec['k']:04d}_{spec['kind']}_N{spec['N']}"
    p.steps = spec["steps"]
    return p


def c5_arrivals(n, mean_gap, seed=None):
    """Poisson arrival times (exponential gaps of the given mean, seconds)
    for a served stream of n requests, seeded (child 0 of the stream's seed)."""
    base = np.random.SeedSequence(BASE_SEED).spawn(5)[4] if seed is None else np.random.SeedSequence(seed)
    rng = np.random.default_rng(base.spawn(1)[0])
    return np.cumsum(rng.exponential(mean_gap, size=n))


def small_case(kind="cylinder", N=48, M=2.0, uncover_mode=UNCOVER_DONOR):
    """Small single instance for parity tests (seconds on the oracle)."""
    p = _body_instance(kind, N, M, uncover_mode=uncover_mode)
    p.name = f"small_{kind}_N{N}"
    return p


def with_state(prob: Problem, Q) -> Problem:
    return replace(prob, Q0=np.asarray(Q, dtype=np.float64))


# ---------------------------------------------------------------------------
# three dimensions: one convex polyhedral body (half-spaces n . x <= c in body
# coordinates) translating at U; Euler with 5 conserved variables
# (rho, rho u, rho v, rho w, E), planes of (nz, ny, nx) cells, x fastest
# ---------------------------------------------------------------------------
@dataclass
class Problem3:
    """One three-dimensional simulation instance."""
    name: str
    nx: int
    ny: int
    nz: int
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    bc: tuple = (TRANSMISSIVE,) * 6          # x-low, x-high, y-low, y-high, z-low, z-high
    gamma: float = GAMMA
    cfl: float = 0.5
    normals: Optional[np.ndarray] = None     # (nplane, 3) outward unit normals
    offsets: Optional[np.ndarray] = None     # (nplane,)
    bbox: tuple = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)   # body bounding box, body coordinates
    U: tuple = (0.0, 0.0, 0.0)
    uncover_mode: int = UNCOVER_DONOR
    Q0: Optional[np.ndarray] = None          # (5, nz, ny, nx)
    info: dict = field(default_factory=dict)

    nc = 5

    @property
    def h(self):
        return tuple((self.hi[a] - self.lo[a]) / (self.nx, self.ny, self.nz)[a] for a in range(3))

    def cell_centres(self):
        c = [self.lo[a] + (np.arange((self.nx, self.ny, self.nz)[a]) + 0.5) * self.h[a] for a in range(3)]
        Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
        return X, Y, Z


def conserved3(rho, u, v, w, p, gamma=GAMMA):
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    u, v, w, p = (np.broadcast_to(np.asarray(a, dtype=np.float64), shape) for a in (u, v, w, p))
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def prism_planes(poly2d):
    """Planes of the z-invariant prism over a convex CCW polygon (n, 2): one
    per edge, normal (ey, -ex, 0) / |e|, offset n . vertex."""
    P = np.asarray(poly2d, dtype=np.float64)
    nrm, off = [], []
    for k in range(len(P)):
        a, b = P[k], P[(k + 1) % len(P)]
        e = b - a
        n = np.array([e[1], -e[0], 0.0]) / math.hypot(e[0], e[1])
        nrm.append(n)
        off.append(float(n[0] * a[0] + n[1] * a[1]))
    return np.array(nrm), np.array(off)


def cone_planes(apex, height, radius, k_sides=24, phase=0.0):
    """A cone along +x (apex forward) as a right pyramid over the regular
    k_sides-gon inscribed in its base circle (vertices at angles 2 pi (m +
    phase) / k_sides): one lateral plane per base edge through the apex, and
    the base plane.  Returns (normals, offsets, bounding box)."""
    ax, ay, az = apex
    xb = ax - height
    A = np.array([ax, ay, az])
    th = 2.0 * math.pi * (np.arange(k_sides) + phase) / k_sides
    V = np.stack([np.full(k_sides, xb), ay + radius * np.cos(th), az + radius * np.sin(th)], axis=1)
    nrm, off = [], []
    for m in range(k_sides):
        n = np.cross(V[m] - A, V[(m + 1) % k_sides] - A)
        mid = 0.5 * (V[m] + V[(m + 1) % k_sides])
        if np.dot(n, mid - np.array([xb, ay, az])) < 0.0:   # outward: away from the axis
            n = -n
        n = n / np.linalg.norm(n)
        nrm.append(n)
        off.append(float(np.dot(n, A)))
    nrm.append(np.array([-1.0, 0.0, 0.0]))
    off.append(-xb)
    bbox = (xb, ax, ay - radius, ay + radius, az - radius, az + radius)
    return np.array(nrm), np.array(off), bbox


N3_MACH = 1.34        # the stationary shock (matches a moving Mach-1.34 shock's jumps)
N3_T_AFTER = 1.48     # 102 us after contact, in tau = D / sqrt(p/rho) of the paper's 20 mm cone


def n3_schardin_cone(cells_per_d=20, k_sides=24, t_after=N3_T_AFTER):
    """The paper's three-dimensional Schardin test (Sec. III.F) as read here,
    in units of the cone's base diameter D and the pre-shock state (rho =
    p = 1): a cone of apex angle 60 deg (an equilateral triangle in
    cross-section), base diameter D, as a right pyramid on a regular
    k_sides-gon, apex along +x, moving with the pre-shock gas at u1 = M c1
    into a stationary Mach-1.34 shock at x = 4 D (the post-shock state from
    the Rankine-Hugoniot relations in the shock's frame); the domain 10 D x
    10 D x 5 D (the paper's 0.2 x 0.2 x 0.1 m), the cone's centre-line on the
    reflective side z = 0 (the paper's half domain), transmissive elsewhere;
    the apex two cells before the shock at t = 0; run until t_after."""
    h = 1.0 / cells_per_d
    g = GAMMA
    c1 = math.sqrt(g)
    u1 = N3_MACH * c1
    r2 = (g + 1.0) * N3_MACH ** 2 / ((g - 1.0) * N3_MACH ** 2 + 2.0)
    p2 = 1.0 + 2.0 * g / (g + 1.0) * (N3_MACH ** 2 - 1.0)
    u2 = u1 / r2
    xs = 4.0 + 0.3183 * h
    H = math.sqrt(3.0) / 2.0
    apex = (xs - 2.0 * h, 0.0 + 0.2718 * h, 0.0)
    # half-step phase: the symmetry plane z = 0 cuts faces through their
    # middles, not along an edge
    n, c, bb = cone_planes(apex, H, 0.5, k_sides, phase=0.5)
    nx, ny, nz = 10 * cells_per_d, 10 * cells_per_d, 5 * cells_per_d
    p = Problem3(f"n3_schardin_cone_{cells_per_d}perD", nx, ny, nz, lo=(0.0, -5.0, 0.0), hi=(10.0, 5.0, 5.0),
                 bc=(TRANSMISSIVE, TRANSMISSIVE, TRANSMISSIVE, TRANSMISSIVE, REFLECTIVE, TRANSMISSIVE),
                 normals=n, offsets=c, bbox=bb, U=(u1, 0.0, 0.0))
    X, Y, Z = p.cell_centres()
    right = X > xs
    p.Q0 = conserved3(np.where(right, r2, 1.0), np.where(right, u2, u1), 0.0, 0.0, np.where(right, p2, 1.0))
    p.info = dict(t_end=t_after, shock_x=xs, post_shock=(r2, u2, p2), u1=u1, cells=nx * ny * nz)
    return p
