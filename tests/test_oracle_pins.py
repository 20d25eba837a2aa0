"""Pins for the parts of the oracle that the whole-sweep invariants do not fix
on their own: the stabilised face flux with shielding from both sides
(Sec. II.C.4, eqs. Klein2DtotalfluxaMethod2 / Klein2shieldedFluxMethod2 and
the two-sided reading), covering and uncovering (Sec. II.C.5, eqs.
volumeWeighting, cutCellInitialisation, cutCellInitialisationDonorCellUpdate,
massDeficitEquation, cutCellCoverDonation), the positivity safeguard, the
Euler branch of the CFL step, and everything rotation touches: the rotated
pose, the wall velocity of a rotating body and the Simpson time average of
the apertures (eq. timeAveragedBeta).

Expected values are worked out by hand from the equations (the working is in
the comments) or come from computations that share nothing with the oracle
(numpy complex rotation, brute-force sampling, finite differences of the
prescribed motion, fine quadrature)."""
import math

import numpy as np
import pytest

import oracle
from paper_1711_11361_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------------------
# stabilised face flux, shielded from one or both sides
# ---------------------------------------------------------------------------
F = np.array([1.0, 2.0, 3.0, 4.0])
FB_L = np.array([0.5, 1.0, -1.0, 2.0])
FB_R = np.array([2.0, 0.0, 1.0, 0.0])


def test_face_one_sided_shielding_by_hand():
    """beta F2D = (beta - s) F + s [FB + d (F - FB)] with s = beta - beta_far.
    beta = 0.8, beta_far = 0.5 -> s = 0.3, d = 0.25:
    0.5 F + 0.3 (0.75 FB + 0.25 F) = 0.575 F + 0.225 FB."""
    got = oracle.stab_face(0.8, F, left=(0.5, 0.25, FB_L))
    assert np.allclose(got, [0.6875, 1.375, 1.5, 2.75], rtol=0, atol=1e-15)
    # the same shielding attached from the right neighbour
    got = oracle.stab_face(0.8, F, right=(0.5, 0.25, FB_L))
    assert np.allclose(got, [0.6875, 1.375, 1.5, 2.75], rtol=0, atol=1e-15)


def test_face_two_sided_within_aperture_by_hand():
    """sL = 0.8 - 0.6 = 0.2 (d 0.25), sR = 0.8 - 0.5 = 0.3 (d 0.5), sum 0.5 <= 0.8:
    0.3 F + 0.3 (0.5 FB_R + 0.5 F) + 0.2 (0.75 FB_L + 0.25 F)
    = 0.5 F + 0.15 FB_R + 0.15 FB_L."""
    got = oracle.stab_face(0.8, F, left=(0.6, 0.25, FB_L), right=(0.5, 0.5, FB_R))
    assert np.allclose(got, [0.875, 1.15, 1.5, 2.3], rtol=0, atol=1e-15)


def test_face_two_sided_clamp_by_hand():
    """Reading for a face shielded from both sides beyond its aperture:
    sL = 0.8 - 0.4 = 0.4, sR = 0.8 - 0.2 = 0.6, sum 1.0 > 0.8, so both scale
    by 0.8: sL = 0.32, sR = 0.48, no unshielded part.
    sR [FB_R + 0.5 (F - FB_R)] = 0.24 (F + FB_R) = [0.72, 0.48, 0.96, 0.96]
    sL [FB_L + 0.25 (F - FB_L)] = 0.24 FB_L + 0.08 F = [0.2, 0.4, 0.0, 0.8]."""
    got = oracle.stab_face(0.8, F, left=(0.4, 0.25, FB_L), right=(0.2, 0.5, FB_R))
    assert np.allclose(got, [0.92, 0.88, 0.96, 1.76], rtol=0, atol=1e-15)


def test_face_far_aperture_larger_gives_no_shielding():
    """A neighbour whose far face is more open than this face shields nothing."""
    got = oracle.stab_face(0.8, F, left=(0.9, 0.25, FB_L), right=(1.0, 0.5, FB_R))
    assert np.array_equal(got, 0.8 * F)


@pytest.mark.parametrize("bfl,bfr,dl,dr", [(0.4, 0.2, 0.25, 0.5), (0.1, 0.0, 0.9, 0.1), (0.7, 0.3, 0.0, 1.0)])
def test_face_consistency_uniform_state(bfl, bfr, dl, dr):
    """When the wall fluxes equal the face flux (a uniform state) the face
    passes beta F whatever the shielding: the weights sum to beta."""
    got = oracle.stab_face(0.8, F, left=(bfl, dl, F), right=(bfr, dr, F))
    assert np.allclose(got, 0.8 * F, rtol=1e-15, atol=0)


# ---------------------------------------------------------------------------
# covering and uncovering
# ---------------------------------------------------------------------------
def _grid3(fill_alpha=1.0, fill_c=7.0):
    return np.full((3, 3), fill_alpha), np.full((1, 3, 3), fill_c)


def test_uncover_donor_by_hand():
    """Centre (1,1) uncovered with alpha_B = 0.2.  Face neighbours at B: west
    alpha 1 (content 2.0), east 0.5 (0.6), south 0.3 (0.5), north solid.
    sigma = 0.2 / (0.2 + 1 + 0.5 + 0.3) = 0.1 (eq. volumeWeighting, the new
    cell counted in the sum); new content 0.1 * (2.0 + 0.6 + 0.5) = 0.31
    (eq. cutCellInitialisation); each donor keeps 0.9 of its content (eq.
    cutCellInitialisationDonorCellUpdate).  Corners are untouched."""
    aB, C = _grid3()
    aB[1, 1], aB[1, 0], aB[1, 2], aB[0, 1], aB[2, 1] = 0.2, 1.0, 0.5, 0.3, 0.0
    aA = aB.copy()
    aA[1, 1] = 0.0
    C[0, 1, 1], C[0, 1, 0], C[0, 1, 2], C[0, 0, 1], C[0, 2, 1] = 0.0, 2.0, 0.6, 0.5, 0.0
    Cn, r, upd = oracle.cover_uncover(aA, aB, C, oracle.UNCOVER_DONOR)
    assert r == 0
    exp = C.copy()
    exp[0, 1, 1], exp[0, 1, 0], exp[0, 1, 2], exp[0, 0, 1] = 0.31, 1.8, 0.54, 0.45
    assert np.allclose(Cn, exp, rtol=0, atol=1e-15)
    assert upd[1, 1] == 1 and upd.sum() == 1
    assert abs(Cn.sum() - C.sum()) < 1e-14


def test_cover_residual_by_hand():
    """Centre covered (alpha 0.1 -> 0) holding 0.9 after the update (eq.
    massDeficitEquation).  Fluid face neighbours at B: west 1, east 0.6,
    south 0.4 (north solid); sum 2.0, so they receive 0.45, 0.27, 0.18
    (eq. cutCellCoverDonation) and the centre ends empty."""
    aB, C = _grid3(fill_c=1.0)
    aB[1, 1], aB[1, 0], aB[1, 2], aB[0, 1], aB[2, 1] = 0.0, 1.0, 0.6, 0.4, 0.0
    aA = aB.copy()
    aA[1, 1] = 0.1
    C[0, 1, 1], C[0, 2, 1] = 0.9, 0.0
    Cn, r, _ = oracle.cover_uncover(aA, aB, C, oracle.UNCOVER_DONOR)
    assert r == 0
    exp = C.copy()
    exp[0, 1, 1], exp[0, 1, 0], exp[0, 1, 2], exp[0, 0, 1] = 0.0, 1.45, 1.27, 1.18
    assert np.allclose(Cn, exp, rtol=0, atol=1e-15)


def test_simultaneous_uncovering_shares_a_donor():
    """Row of five cells: (1) and (3) uncovered (alpha_B 0.5), the others fluid
    with alpha 1 and content 1; rows above and below solid.  Each new cell
    has sigma = 0.5 / 2.5 = 0.2 and takes 0.2 * 2 = 0.4; the shared donor
    (2) loses 0.2 to each, as both events read the contents before any of
    them (order-free), ending at 0.6; cells (0) and (4) end at 0.8."""
    aB = np.zeros((3, 5))
    aB[1] = [1.0, 0.5, 1.0, 0.5, 1.0]
    aA = aB.copy()
    aA[1, 1] = aA[1, 3] = 0.0
    C = np.zeros((1, 3, 5))
    C[0, 1] = [1.0, 0.0, 1.0, 0.0, 1.0]
    Cn, r, _ = oracle.cover_uncover(aA, aB, C, oracle.UNCOVER_DONOR)
    assert r == 0
    assert np.allclose(Cn[0, 1], [0.8, 0.4, 0.6, 0.4, 0.8], rtol=0, atol=1e-15)
    assert abs(Cn.sum() - 3.0) < 1e-14


def test_uncovered_neighbour_is_no_donor_and_diagonal_fallback():
    """An uncovered neighbour has no content yet and donates nothing.  The
    centre (alpha_B 0.1) and its east neighbour (alpha_B 0.4) are both newly
    uncovered; the only other fluid cell is the north-east corner (alpha 0.9,
    content 1.0).  The centre has no face neighbour left to take from (its
    east neighbour is new) and falls back to its 8-neighbourhood (a
    reading): sigma = 0.1 / (0.1 + 0.9) = 0.1.  The east cell has the corner
    as its north face neighbour: sigma = 0.4 / (0.4 + 0.9) = 0.4 / 1.3.  Both
    read the corner's content from before either event."""
    aB = np.zeros((3, 3))
    aB[1, 1], aB[1, 2], aB[2, 2] = 0.1, 0.4, 0.9
    aA = aB.copy()
    aA[1, 1] = aA[1, 2] = 0.0
    C = np.zeros((1, 3, 3))
    C[0, 2, 2] = 1.0
    Cn, r, _ = oracle.cover_uncover(aA, aB, C, oracle.UNCOVER_DONOR)
    assert r == 0
    s_centre, s_east = 0.1, 0.4 / 1.3
    assert abs(Cn[0, 1, 1] - s_centre * 1.0) < 1e-15
    assert abs(Cn[0, 1, 2] - s_east * 1.0) < 1e-15
    assert abs(Cn[0, 2, 2] - (1.0 - s_centre - s_east)) < 1e-15
    assert abs(Cn.sum() - 1.0) < 1e-15


def test_flux_gcl_mode_leaves_uncovered_cells_to_the_update():
    """In the flux-GCL mode an uncovered cell fills through its swept
    apertures, so the redistribution leaves it alone; covering still acts."""
    aB, C = _grid3(fill_c=1.0)
    aB[1, 1] = 0.3
    aA = aB.copy()
    aA[1, 1] = 0.0
    aB[0, 0] = 0.0        # corner (0,0) covered: content 0.5 to (0,1) and (1,0)
    C[0, 0, 0] = 0.5
    C[0, 1, 1] = 0.123
    Cn, r, upd = oracle.cover_uncover(aA, aB, C, oracle.UNCOVER_FLUX_GCL)
    assert r == 0 and upd.sum() == 0
    assert Cn[0, 1, 1] == 0.123
    assert Cn[0, 0, 0] == 0.0
    assert abs(Cn[0, 0, 1] - 1.25) < 1e-15 and abs(Cn[0, 1, 0] - 1.25) < 1e-15


def test_covered_cell_on_an_open_side_passes_its_residual_out():
    """A body leaving through a transmissive side: the covered cell in the
    last column has no fluid neighbour left, so its residual (0.7) leaves
    the domain instead of failing the sweep; on a closed side it fails."""
    aA = np.zeros((3, 3))
    aA[1, 2] = 0.3
    aB = np.zeros((3, 3))
    C = np.zeros((1, 3, 3))
    C[0, 1, 2] = 0.7
    Cn, r, _ = oracle.cover_uncover(aA, aB, C, oracle.UNCOVER_DONOR, open_sides=2)
    assert r == 0 and Cn[0, 1, 2] == 0.0 and Cn.sum() == 0.0
    _, r, _ = oracle.cover_uncover(aA, aB, C, oracle.UNCOVER_DONOR, open_sides=1)
    assert r == -4


def test_event_without_any_fluid_neighbour_is_reported():
    aB = np.zeros((3, 3))
    aB[1, 1] = 0.5
    aA = np.zeros((3, 3))
    Cn, r, _ = oracle.cover_uncover(aA, aB, np.zeros((1, 3, 3)), oracle.UNCOVER_DONOR)
    assert r == -4


# ---------------------------------------------------------------------------
# positivity safeguard
# ---------------------------------------------------------------------------
def _euler(nx, ny, rho=1.0, E=2.5):
    C = np.zeros((4, ny, nx))
    C[0], C[3] = rho, E
    return C


def test_safeguard_one_merge_by_hand():
    """Centre (alpha 0.5) holds rho = -0.1 (E 0.1): non-physical.  It merges
    with its four face neighbours (alpha 1, rho 1, E 2.5): total rho 3.9,
    E 10.1, volume 4.5, shared by volume: rho = 3.9/4.5 * alpha,
    E = 10.1/4.5 * alpha.  Corners are not in the cluster."""
    a = np.ones((3, 3))
    a[1, 1] = 0.5
    C = _euler(3, 3)
    C[:, 1, 1] = [-0.1, 0.0, 0.0, 0.1]
    Cn, m = oracle.safeguard(a, C)
    assert m == 5
    for (j, i) in [(1, 0), (1, 2), (0, 1), (2, 1)]:
        assert abs(Cn[0, j, i] - 3.9 / 4.5) < 1e-15 and abs(Cn[3, j, i] - 10.1 / 4.5) < 1e-15
    assert abs(Cn[0, 1, 1] - 0.5 * 3.9 / 4.5) < 1e-15 and abs(Cn[3, 1, 1] - 0.5 * 10.1 / 4.5) < 1e-15
    for (j, i) in [(0, 0), (0, 2), (2, 0), (2, 2)]:
        assert Cn[0, j, i] == 1.0 and Cn[3, j, i] == 2.5


def test_safeguard_second_merge_by_hand():
    """Centre of a 5x5 grid with rho = -10 (E 1), all others rho 1, E 2.5,
    alpha 1.  First merge (centre + 4): rho = -6/5 each, still bad, E 11/5.
    Second merge: those five plus their eight further face neighbours,
    13 cells: rho = (-6 + 8)/13, E = (11 + 20)/13.  Cells merged: 5 + 13."""
    a = np.ones((5, 5))
    C = _euler(5, 5)
    C[:, 2, 2] = [-10.0, 0.0, 0.0, 1.0]
    Cn, m = oracle.safeguard(a, C)
    assert m == 18
    cluster = [(2, 2), (1, 2), (3, 2), (2, 1), (2, 3), (0, 2), (4, 2), (2, 0), (2, 4), (1, 1), (1, 3), (3, 1), (3, 3)]
    for (j, i) in cluster:
        assert abs(Cn[0, j, i] - 2.0 / 13.0) < 1e-15 and abs(Cn[3, j, i] - 31.0 / 13.0) < 1e-14
    for (j, i) in [(0, 0), (0, 1), (4, 4), (1, 0)]:
        assert Cn[0, j, i] == 1.0
    assert abs(Cn[0].sum() - C[0].sum()) < 1e-13 and abs(Cn[3].sum() - C[3].sum()) < 1e-13


def test_safeguard_leaves_physical_contents_alone():
    a = np.ones((4, 4))
    C = _euler(4, 4)
    Cn, m = oracle.safeguard(a, C)
    assert m == 0 and np.array_equal(Cn, C)


def _collapsed(aA_c, aB_c):
    """3x3, the centre's volume fraction goes from aA_c to aB_c in the sweep
    and it holds a physical but far out-of-range state (rho 50, E 125); the
    others alpha 1, rho 1, E 2.5."""
    aA, aB = np.ones((3, 3)), np.ones((3, 3))
    aA[1, 1], aB[1, 1] = aA_c, aB_c
    C = _euler(3, 3)
    C[:, 1, 1] = [50.0 * aB_c, 0.0, 0.0, 125.0 * aB_c]
    return aA, aB, C


def test_safeguard_collapsed_cell_merges_by_hand():
    """alpha 0.5 -> 0.004 keeps 0.8% of the volume: the centre seeds the
    first merge although its state is physical.  Cluster: centre + 4 face
    neighbours, rho total 0.2 + 4, E total 0.5 + 10, volume 4.004."""
    aA, aB, C = _collapsed(0.5, 0.004)
    Cn, m = oracle.safeguard(aB, C, alphaA=aA)
    assert m == 5
    for (j, i) in [(1, 0), (1, 2), (0, 1), (2, 1)]:
        assert abs(Cn[0, j, i] - 4.2 / 4.004) < 1e-15 and abs(Cn[3, j, i] - 10.5 / 4.004) < 1e-14
    assert abs(Cn[0, 1, 1] - 0.004 * 4.2 / 4.004) < 1e-17
    assert Cn[0, 0, 0] == 1.0
    assert abs(Cn[0].sum() - C[0].sum()) < 1e-14 and abs(Cn[3].sum() - C[3].sum()) < 1e-14


def test_safeguard_collapse_threshold_and_exclusions():
    """1% of the start volume is the boundary: alpha 0.5 -> 0.0051 is left
    alone; without the start fractions, or for a cell uncovered in the
    sweep (alpha 0 -> 0.001), nothing is seeded; a physical collapsed cell
    seeds the first merge only (one merge of 5 cells, not one per layer)."""
    aA, aB, C = _collapsed(0.5, 0.0051)
    assert oracle.safeguard(aB, C, alphaA=aA)[1] == 0
    aA, aB, C = _collapsed(0.5, 0.004)
    assert oracle.safeguard(aB, C)[1] == 0
    aA, aB, C = _collapsed(0.0, 0.001)
    assert oracle.safeguard(aB, C, alphaA=aA)[1] == 0
    aA, aB, C = _collapsed(0.9, 0.0001)
    assert oracle.safeguard(aB, C, alphaA=aA)[1] == 5


def test_collapse_sweep_keeps_uniform_flow_uniform():
    """A whole column goes from alpha 0.3 to 0.002 in one x sweep (the slab
    of inputs.collapse_slab): its cells seed merges, and gas moving with the
    slab stays uniform (the stabilised update keeps uniform flow, and merging
    equal states changes nothing)."""
    prob = inputs.collapse_slab(uniform=True)
    o = oracle.Oracle(prob)
    a0 = o.alpha()
    assert np.all(np.abs(a0[10:22, 19] - 0.3) < 1e-12)
    assert o.sweep(0, inputs.COLLAPSE_SLAB_DT) == 0
    a1 = o.alpha()
    assert np.all(np.abs(a1[10:22, 19] - 0.002) < 1e-12)
    assert o.last_sweep()[1] >= 12
    Q = o.state()
    fl = a1 > 0
    for q, v in enumerate((1.0, 1.0, 0.0, 1.0 / 0.4 + 0.5)):
        assert np.max(np.abs(Q[q][fl] - v)) < 1e-12, q


# ---------------------------------------------------------------------------
# CFL step, Euler branch (regular-cell wave speeds, raised to the wall speed)
# ---------------------------------------------------------------------------
def _cfl_problem(U=(0.0, 0.0), rot=None):
    """40 x 10 cells on the unit square (dx = 0.025, dy = 0.1), CFL 0.5."""
    nx, ny = 40, 10
    polys, mov, piv, a1, om = [], [], (0.5, 0.5), 0.0, 0.0
    if rot is not None:
        polys = [inputs.rect_polygon(0.4, 0.4, 0.6, 0.6)]
        mov = [1]
        a1, om = rot
    elif U != (0.0, 0.0):
        polys = [inputs.rect_polygon(0.41, 0.41, 0.59, 0.59)]
        mov = [1]
    p = inputs.Problem("cfl", nx, ny, 0.0, 0.0, 1.0, 1.0, cfl=0.5, polygons=polys, moving=mov, U=U, pivot=piv,
                       a1=a1, omega=om)
    # gas at rest with c = 1 (rho 1, p 1/1.4), one cell moving at (0.5, -2)
    rho = np.ones((ny, nx))
    u = np.zeros((ny, nx))
    v = np.zeros((ny, nx))
    u[3, 5], v[3, 5] = 0.5, -2.0
    p.Q0 = inputs.conserved(rho, u, v, np.full((ny, nx), 1.0 / 1.4))
    return p


def test_cfl_dt_by_hand():
    """S_x = max(|u| + c) = 1.5, S_y = 3; CFL 0.5:
    dt = 0.5 * min(0.025/1.5, 0.1/3) = 0.5 / 60 = 1/120."""
    assert abs(oracle.Oracle(_cfl_problem()).cfl_dt() - 1.0 / 120.0) < 1e-17


def test_cfl_dt_raised_to_body_speed_by_hand():
    """A body translating at (4, 0) raises S_x to 4:
    dt = 0.5 * min(0.025/4, 0.1/3) = 0.003125."""
    assert abs(oracle.Oracle(_cfl_problem(U=(4.0, 0.0))).cfl_dt() - 0.003125) < 1e-17


def test_cfl_dt_raised_to_rotation_speed_by_hand():
    """A square of half-side 0.1 about its centre, theta = sin(30 t): the
    largest wall speed is |a1 omega| r_max = 30 * 0.1 sqrt(2) = 4.2426...,
    above both fluid speeds: dt = 0.5 * 0.025 / 4.2426... = 0.0029462782..."""
    got = oracle.Oracle(_cfl_problem(rot=(1.0, 30.0))).cfl_dt()
    assert abs(got - 0.0125 / (3.0 * math.sqrt(2.0))) < 1e-16


# ---------------------------------------------------------------------------
# rotation: pose, wall velocity, Simpson average of the apertures
# ---------------------------------------------------------------------------
def _rotate_np(poly, pivot, theta, shift=(0.0, 0.0)):
    """Rotate by theta about pivot, then translate (numpy complex arithmetic)."""
    z = poly[:, 0] + 1j * poly[:, 1]
    c = complex(*pivot)
    w = c + np.exp(1j * theta) * (z - c) + complex(*shift)
    return np.stack([w.real, w.imag], axis=1)


def _inside(poly, X, Y):
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


def _rot_problem(N=32, pivot=(0.47, 0.52), a0=0.0, a1=1.0, omega=1.0, U=(0.0, 0.0), body="naca"):
    if body == "naca":
        poly = inputs.naca00xx_polygon(chord=0.6, n_side=41, le=(0.2, 0.52))
    else:
        h = 0.2371     # sides off the grid lines of every grid used here
        poly = inputs.rect_polygon(0.5 - h, 0.5 - h, 0.5 + h, 0.5 + h)
    p = inputs.Problem("rot", N, N, 0.0, 0.0, 1.0, 1.0, bc=(0, 0, 0, 0), cfl=0.5, polygons=[poly], moving=[1],
                       U=U, pivot=pivot, a0=a0, a1=a1, omega=omega)
    X, Y = p.cell_centres()
    p.Q0 = inputs.conserved(np.ones_like(X), 0.0, 0.0, 1.0)
    return p, poly


@pytest.mark.parametrize("theta,shift", [(0.3, (0.0, 0.0)), (-0.7, (0.031, -0.02)), (2.4, (0.0, 0.05))])
def test_rotated_pose_equals_independently_rotated_polygon(theta, shift):
    """The oracle's geometry at pose (X, Y, theta) equals its geometry at the
    identity pose of the polygon rotated about the pivot and shifted in
    numpy, to round-off (pins the sense of rotation, the pivot and the order
    rotate-then-translate), and brute-force sampling of that polygon."""
    p, poly = _rot_problem(N=24)
    a, t, bx, by = oracle.Oracle(p).geometry(shift[0], shift[1], theta)
    q = _rotate_np(poly, p.pivot, theta, shift)
    p2 = inputs.Problem("rot2", p.nx, p.ny, 0.0, 0.0, 1.0, 1.0, polygons=[q], moving=[1])
    a2, t2, bx2, by2 = oracle.Oracle(p2).geometry()
    assert np.max(np.abs(a - a2)) < 1e-13
    assert np.max(np.abs(bx - bx2)) < 1e-13 and np.max(np.abs(by - by2)) < 1e-13
    s = 64
    off = (np.arange(s) + 0.5) / s
    for j in range(p.ny):
        for i in range(p.nx):
            if not t[j, i]:
                continue
            X, Y = np.meshgrid(p.x0 + (i + off) * p.dx, p.y0 + (j + off) * p.dy)
            assert abs(a[j, i] - (1.0 - _inside(q, X, Y).mean())) <= 4.0 / s


@pytest.mark.parametrize("step_sweeps", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_wall_velocity_of_rotation_equals_finite_difference(step_sweeps):
    """Rotation about a fixed pivot, theta(t) = a0 + a1 sin(omega t).  The
    wall velocity the sweep uses at a band cell is the velocity, at the
    sweep's mid time, of the body point that sits at the cell centre then:
    a central finite difference of the prescribed motion of that material
    point (numpy), to O(h^2)."""
    step, sweep = step_sweeps
    p, _ = _rot_problem(N=32, a0=0.1, a1=0.8, omega=3.0)
    o = oracle.Oracle(p)
    dt = 0.01
    order = []
    for k in range(step + 1):
        order = (0, 1) if k % 2 == 0 else (1, 0)
        for m, d in enumerate(order):
            assert o.sweep(d, dt) == 0
            if k == step and m == sweep:
                break
    wall = o.last_wall()
    t0 = step * dt
    tM = t0 + (0.25 if sweep == 0 else 0.75) * dt
    theta = lambda t: 0.1 + 0.8 * math.sin(3.0 * t)
    c = complex(*p.pivot)
    xc, yc = p.cell_centres()
    has = wall["has"] > 0
    assert has.sum() > 20
    h = 1e-5
    zc = xc[has] + 1j * yc[has]
    z0 = c + np.exp(-1j * theta(tM)) * (zc - c)          # material point at the cell centre at tM
    vel = (np.exp(1j * theta(tM + h)) - np.exp(1j * theta(tM - h))) * (z0 - c) / (2 * h)
    assert np.max(np.abs(wall["wx"][has] - vel.real)) < 1e-8
    assert np.max(np.abs(wall["wy"][has] - vel.imag)) < 1e-8


def test_wall_velocity_of_translation_and_rotation():
    """A translating, rotating body: the wall velocity is the body velocity U
    plus the rotation about the pivot carried with the body (at the sweep's
    mid pose, to which the x sweep has moved the body by half of U_x dt)."""
    U = (0.3, -0.2)
    p, _ = _rot_problem(N=32, a0=0.0, a1=0.5, omega=2.0, U=U)
    o = oracle.Oracle(p)
    dt = 0.01
    assert o.sweep(0, dt) == 0
    wall = o.last_wall()
    tM = 0.25 * dt
    om = 0.5 * 2.0 * math.cos(2.0 * tM)            # d theta / dt at tM (derivative of the prescribed motion)
    piv = complex(p.pivot[0] + 0.5 * U[0] * dt, p.pivot[1])
    xc, yc = p.cell_centres()
    has = wall["has"] > 0
    r = xc[has] + 1j * yc[has] - piv
    vel = complex(*U) + 1j * om * r
    assert np.max(np.abs(wall["wx"][has] - vel.real)) < 1e-14
    assert np.max(np.abs(wall["wy"][has] - vel.imag)) < 1e-14


def _time_average_error(dt, N=64):
    """Max over smooth faces of |beta_tilde - (1/dt_s) int beta dt| for the first
    x sweep (rotation from theta(0) to theta(dt/2)) of a square rotating about
    its centre, against composite Simpson with 256 panels of the oracle's
    instantaneous apertures (pinned by brute force elsewhere)."""
    p, poly = _rot_problem(N=N, pivot=(0.5, 0.5), a0=0.0, a1=1.0, omega=1.0, body="square")
    o = oracle.Oracle(p)
    assert o.sweep(0, dt) == 0
    d, bt = o.last_faces()
    assert d == 0
    ts = np.linspace(0.0, 0.5 * dt, 257)
    geo = oracle.Oracle(p)
    samples = np.stack([geo.geometry(0.0, 0.0, math.sin(t))[2] for t in ts])
    w = np.ones(257)
    w[1:-1:2], w[2:-1:2] = 4.0, 2.0
    ref = np.tensordot(w, samples, axes=1) / (3.0 * 256)
    # smooth faces: one straight edge crosses the face at every sample (the
    # aperture stays strictly inside (0, 1)) and no vertex comes near
    inner = np.all((samples > 0.0) & (samples < 1.0), axis=0)
    verts = np.concatenate([_rotate_np(poly, (0.5, 0.5), math.sin(t)) for t in (0.0, 0.25 * dt, 0.5 * dt)])
    yf = (np.arange(N) + 0.5) / N
    xf = np.arange(N + 1) / N
    XF, YF = np.meshgrid(xf, yf)
    far = np.ones_like(inner)
    for vx, vy in verts:
        far &= (np.abs(XF - vx) > 2.0 / N) | (np.abs(YF - vy) > 2.0 / N)
    sel = inner & far
    assert sel.sum() >= 20
    return np.max(np.abs(bt - ref)[sel])


def test_simpson_time_averaged_aperture_converges_at_fourth_order():
    """eq. timeAveragedBeta is the time average of the aperture over the
    sweep; for rotation the oracle takes Simpson's rule over the poses A,
    mid and B (reading).  Against a fine quadrature its error falls by about
    16 when the sweep's time step halves (trapezoid or midpoint weights, or
    a pose taken at the wrong time, would give 4 or less)."""
    e1 = _time_average_error(0.08)
    e2 = _time_average_error(0.04)
    assert e1 < 1e-6
    assert e1 / e2 > 10.0, (e1, e2)
