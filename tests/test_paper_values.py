"""The paper's printed values under tests/golden/ and the host post-processing that
the GPU physics tests compare against them, pinned without a GPU:

  * the analytical Moffatt ratios of Tables 1 and 2 (triangular cavity flow, Sec. 5)
    follow from the corner eigenvalue of Stokes flow in the printed wedge angle;
  * the printed apex angle is that of the triangle of base 1 and height 2 that the
    printed node count (400 x 800 / 2) samples;
  * the force probe (tests/forces.py) gives the closed-form force of polynomial
    fields on the circular cylinder of the drag tests, with the oracle's MLS
    derivative tables standing in for the GPU's;
  * the Strouhal estimator recovers the frequency of a synthetic lift signal
    sampled like the shedding test's.
"""
import math

import numpy as np
import pytest

import workloads as w
from forces import ForceProbe, strouhal
from oracle import vip_oracle as vo
from paper_values import load


# -- Moffatt eddies ------------------------------------------------------------

def corner_eigenvalue(two_alpha):
    """Exponent lambda of the dominant eddy mode psi = r^lambda f(theta) of Stokes
    flow in a wedge |theta| <= alpha, psi even in theta (the flow that a lid far
    from the corner drives).

    f = A cos(lambda theta) + C cos((lambda - 2) theta) with f = f' = 0 on both
    walls has a non-zero (A, C) only where
        (lambda - 2) cos(lambda alpha) sin((lambda - 2) alpha)
          - lambda sin(lambda alpha) cos((lambda - 2) alpha) = 0,
    which with p = lambda - 1 and the product-to-sum identities reads
        g(p) = sin(2 p alpha) + p sin(2 alpha) = 0.
    g is odd, so roots come in pairs +-p; the velocity ~ r^(Re p) vanishes at the
    corner only for Re p > 0.  Complex roots (Im p > 0) give eddies; the dominant
    one has the smallest real part.  Roots found by Newton's method from a grid of
    starting points."""
    a = 0.5 * two_alpha
    with np.errstate(all="ignore"):  # starts that wander off overflow harmlessly
        roots = _newton_roots(a)
    assert roots
    p = min(roots, key=lambda z: z.real)
    return p + 1.0


def _newton_roots(a):
    roots = []
    for re0 in np.arange(1.0, 30.0, 0.5):
        for im0 in np.arange(0.25, 12.0, 0.5):
            p = complex(re0, im0)
            for _ in range(100):
                if not abs(p) < 1e3:  # left the region of interest
                    break
                g = np.sin(2 * p * a) + p * np.sin(2 * a)
                dg = 2 * a * np.cos(2 * p * a) + np.sin(2 * a)
                step = g / dg
                p -= step
                if abs(step) < 1e-14 * abs(p):
                    break
            g = np.sin(2 * p * a) + p * np.sin(2 * a)
            if abs(g) < 1e-10 * max(1.0, abs(p)) and p.imag > 1e-6 and p.real > 0:
                roots.append(p)
    return roots


def test_moffatt_ratios_follow_from_the_corner_eigenvalue():
    """Between consecutive sign changes of Re(r^(i Im lambda)) ln r moves by
    pi / Im lambda, so r_n / r_(n+1) = exp(pi / Im lambda); the velocity scales as
    r^(Re lambda - 1), so I_n / I_(n+1) = exp(pi (Re lambda - 1) / Im lambda).  The
    paper prints both to three significant digits."""
    g = load("moffatt_wedge.txt")
    lam = corner_eigenvalue(math.radians(g["apex_angle_deg"]))
    r_ratio = math.exp(math.pi / lam.imag)
    i_ratio = math.exp(math.pi * (lam.real - 1.0) / lam.imag)
    assert abs(r_ratio - g["moffatt.r_ratio"]) <= 0.005, r_ratio
    assert abs(i_ratio - g["moffatt.I_ratio"]) <= 0.5, i_ratio


@pytest.mark.parametrize("two_alpha_deg", [28.072, 60.0, 90.0])
def test_corner_eigenvalue_solves_the_wall_conditions(two_alpha_deg):
    """The root makes the 2x2 determinant of the wall conditions vanish, in its form
    before the product-to-sum step; a narrower wedge packs its eddies closer
    (larger Im lambda, smaller r_n / r_(n+1))."""
    two_alpha = math.radians(two_alpha_deg)
    lam = corner_eigenvalue(two_alpha)
    a = 0.5 * two_alpha
    det = ((lam - 2) * np.cos(lam * a) * np.sin((lam - 2) * a)
           - lam * np.sin(lam * a) * np.cos((lam - 2) * a))
    scale = abs(lam) * max(1.0, abs(np.cos(lam * a)) * abs(np.sin((lam - 2) * a)))
    assert abs(det) <= 1e-9 * scale, det
    assert lam.real > 1.0 and lam.imag > 0.0
    if two_alpha_deg < 90.0:
        assert lam.imag > corner_eigenvalue(math.radians(90.0)).imag


def test_apex_angle_is_the_base_1_height_2_triangle():
    g = load("moffatt_wedge.txt")
    nx, ny = g["nodes"]
    # 400 x 800 / 2 nodes: a lattice twice as tall as it is wide, halved by the
    # triangle; its apex half-angle is atan((1/2) / 2)
    assert ny == 2 * nx
    assert round(math.degrees(2 * math.atan(0.5 / 2.0)), 3) == g["apex_angle_deg"]


def test_vip_rows_within_the_paper_s_agreement():
    """Transcription check of the computed rows: the paper calls the agreement good;
    every stored ratio is within 3 % (distances) and 7 % (intensities) of Moffatt's."""
    g = load("moffatt_wedge.txt")
    assert len(g["vip.r_ratio"]) == len(g["vip.I_ratio"]) == 5
    for r in g["vip.r_ratio"]:
        assert abs(r / g["moffatt.r_ratio"] - 1.0) <= 0.03, r
    for i in g["vip.I_ratio"]:
        assert abs(i / g["moffatt.I_ratio"] - 1.0) <= 0.07, i


# -- cylinder table and its post-processing --------------------------------------

def test_cylinder_table_fixture():
    t = load("cylinder_table.txt")
    assert set(t) == {"Re40.C_D", "Re100.C_D", "Re100.CL_amp", "Re100.St"}
    assert t["Re40.C_D"] > t["Re100.C_D"] > 1.0
    assert 0.1 < t["Re100.St"] < 0.25 and 0.0 < t["Re100.CL_amp"] < 1.0


class FieldContext:
    """Stand-in for a solver context: the oracle's MLS derivative tables (D10, D01)
    on the rows of the body's surface nodes, and a prescribed state."""

    def __init__(self, ns, rows, u, v, p):
        self.n = ns.n
        rho = 2.2 * ns.h[rows]
        qptr, qidx = vo.neighbours(ns.x[rows], ns.y[rows], rho, ns.x, ns.y, ns.Lx, ns.Ly)
        wts = vo.mls_weights(ns.x[rows], ns.y[rows], rho, qptr, qidx, ns.x, ns.y, ns.Lx, ns.Ly,
                             "cubic_spline", derivs=((1, 0), (0, 1)))
        counts = np.zeros(ns.n, np.int64)
        counts[rows] = np.diff(qptr)
        order = np.argsort(rows, kind="stable")
        self.ptr = np.concatenate([[0], np.cumsum(counts)])
        seg = [np.arange(qptr[k], qptr[k + 1]) for k in order]
        sel = np.concatenate(seg)
        self.col = qidx[sel]
        self.tab = {"D10": wts[(1, 0)][sel], "D01": wts[(0, 1)][sel]}
        self.state = (u, v, p, np.zeros(ns.n))

    def vip_get_stencil(self, which):
        return self.ptr, self.col, self.tab[which]

    def vip_get_state(self):
        return self.state


@pytest.fixture(scope="module")
def cylinder():
    # the drag tests' body and spacing on a smaller channel (the probe's surface test
    # r < 2 must not reach the inlet wall at x = -3)
    return w.channel_body(1 / 16, ("circle", 0.5), Re=40.0, xlim=(-3.0, 4.0), ylim=(-3.0, 3.0))


CASES = {
    # name: (u coefficients, v coefficients, p coefficients) on the monomials
    # [1, x, y, x^2, x y, y^2] (p linear)
    "pressure_x": ([0] * 6, [0] * 6, [0.0, 1.0, 0.0]),
    "pressure_y": ([0] * 6, [0] * 6, [0.0, 0.0, 1.0]),
    "shear_u_y2": ([0, 0, 0, 0, 0, 1.0], [0] * 6, [0.0, 0.0, 0.0]),
    "shear_v_x2": ([0] * 6, [0, 0, 0, 1.0, 0, 0], [0.0, 0.0, 0.0]),
    "mixed": ([0.3, -0.7, 0.2, 0.9, -0.4, 0.6], [-0.1, 0.5, 0.8, -0.3, 0.7, -0.2], [0.4, -1.1, 0.6]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_force_probe_closed_forms(cylinder, case):
    """Force on the body F = (closed surface) sum of sigma n ds with
    sigma = -p I + (1/Re)(grad u + grad u^T).  For polynomial fields the divergence
    theorem over the disc of radius R gives F = pi R^2 div sigma, and for linear p
    and quadratic (u, v), with u = a0 + ax x + ay y + axx x^2 + axy x y + ayy y^2 and v
    likewise with b,
        div sigma = -grad p + (1/Re) (lap u + grad div u)
                  = (-p_x + (4 axx + 2 ayy + bxy) / Re,  -p_y + (2 bxx + 4 byy + axy) / Re),
    a constant.  C = 2 F.  The probe sums over M surface nodes equally spaced in
    angle with ds = (polygon perimeter) / M: the trigonometric integrands are summed
    exactly, and ds = 2 pi R / M times sin(pi/M) / (pi/M)."""
    ns = cylinder
    a, b, pc = (np.asarray(c, float) for c in CASES[case])
    x, y = ns.x, ns.y
    mono = np.stack([np.ones_like(x), x, y, x * x, x * y, y * y])
    u, v = a @ mono, b @ mono
    p = pc[0] + pc[1] * x + pc[2] * y
    r = np.hypot(x, y)
    s = np.nonzero((ns.kind == vo.KIND_WALL) & (r < 2.0))[0]
    M = s.size
    th = np.sort(np.arctan2(y[s], x[s]))
    assert np.allclose(np.diff(th), 2 * np.pi / M, atol=1e-9, rtol=0)
    R = 0.5
    assert np.allclose(r[s], R, atol=1e-12, rtol=0)
    Re = ns.Re
    div_sigma = np.array([-pc[1] + (4 * a[3] + 2 * a[5] + b[4]) / Re,
                          -pc[2] + (2 * b[3] + 4 * b[5] + a[4]) / Re])
    kappa = math.sin(math.pi / M) / (math.pi / M)
    expect = 2 * math.pi * R * R * div_sigma * kappa
    probe = ForceProbe(FieldContext(ns, s, u, v, p), ns)
    cd, cl = probe.coefficients()
    assert abs(cd - expect[0]) <= 1e-9 * (1 + abs(expect[0])), (cd, expect)
    assert abs(cl - expect[1]) <= 1e-9 * (1 + abs(expect[1])), (cl, expect)


def test_strouhal_estimator_on_synthetic_lift():
    """Sampling of the shedding test (h = 1/16, dt = h/4, every 6 steps over 40 time
    units); a sinusoid with an offset and a weak second harmonic, frequencies across
    the Re = 100 range, random phases: within 0.5 % (the test's bar on St is 3 %)."""
    dt = 0.25 / 16
    k = int(round(0.1 / dt))
    n = int(round(40.0 / (k * dt)))
    t = (np.arange(n) + 1) * k * dt
    rng = np.random.default_rng(164)
    for f in np.linspace(0.14, 0.19, 11):
        for ph in rng.uniform(0.0, 2 * np.pi, 3):
            cl = 0.02 + 0.31 * np.sin(2 * np.pi * f * t + ph) + 0.01 * np.sin(4 * np.pi * f * t + 2 * ph)
            assert abs(strouhal(t, cl) / f - 1.0) <= 5e-3, (f, ph)


# -- bumpy cylinders ---------------------------------------------------------------

def test_bumpy_fixture_is_consistent():
    g = load("bumpy_drag.txt")
    assert g["m_b"] == [10.0 * k for k in range(1, 11)]
    # the characteristic length is the body's largest radius
    assert math.isclose(g["R"], g["r0"] * (1 + g["gamma"]), rel_tol=1e-12)
    assert g["cd_peak_m_b"] in g["m_b"] and 0.0 < g["cd_reduction_min"] < 1.0


def test_force_probe_on_a_bumpy_body_is_second_order():
    """On the body r = r0 (1 + gamma cos(m_b theta)) (m_b = 10) the probe's sum over
    surface nodes at equal arc length is a quadrature of second order in h: for a
    mixed polynomial field its force approaches the divergence-theorem value
    (area pi r0^2 (1 + gamma^2 / 2)) with error ratio ~4 when h halves."""
    g = load("bumpy_drag.txt")
    r0, gamma = g["r0"], g["gamma"]
    a, b, pc = (np.asarray(c, float) for c in CASES["mixed"])
    errs = []
    for h in (1 / 32, 1 / 64):
        ns = w.channel_body(h, ("bumps", r0, gamma, 10), Re=g["Re"], xlim=(-3.0, 4.0), ylim=(-3.0, 3.0))
        x, y = ns.x, ns.y
        mono = np.stack([np.ones_like(x), x, y, x * x, x * y, y * y])
        s = np.nonzero((ns.kind == vo.KIND_WALL) & (np.hypot(x, y) < 2.0))[0]
        probe = ForceProbe(FieldContext(ns, s, a @ mono, b @ mono, pc[0] + pc[1] * x + pc[2] * y), ns)
        cd, cl = probe.coefficients()
        area = math.pi * r0 * r0 * (1 + gamma * gamma / 2)
        div_sigma = np.array([-pc[1] + (4 * a[3] + 2 * a[5] + b[4]) / ns.Re,
                              -pc[2] + (2 * b[3] + 4 * b[5] + a[4]) / ns.Re])
        expect = 2 * area * div_sigma
        errs.append(max(abs(cd / expect[0] - 1), abs(cl / expect[1] - 1)))
    assert errs[0] < 6e-3 and errs[1] < 1.5e-3, errs
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


# -- the Moffatt cavity as a workload ------------------------------------------------

def test_wedge_cavity_samples_the_printed_triangle():
    """workloads.wedge_cavity is the triangle of Tables 1-2: apex angle 28.072
    degrees, every node in the closed triangle, wall nodes on its edges with unit
    normals pointing out of it, and about (n_base - 1)^2 nodes (the area is 1 in
    units of the base), as 400 x 800 / 2 is for a 400-node base."""
    g = load("moffatt_wedge.txt")
    ns = w.wedge_cavity(49)
    h = ns.meta["h"]
    assert round(ns.meta["apex_angle_deg"], 3) == g["apex_angle_deg"]
    x, y = ns.x, ns.y
    # inside: below the lid, right of the left edge, left of the right edge
    L = math.hypot(0.5, 2.0)
    dl = (2.0 * x - 0.5 * (-y)) / L          # distance from the left edge, inwards
    dr = (2.0 * (1.0 - x) - 0.5 * (-y)) / L  # from the right edge
    assert np.all(y <= 1e-12) and np.all(dl >= -1e-12) and np.all(dr >= -1e-12)
    wall = ns.kind == vo.KIND_WALL
    on_edge = (np.abs(y) < 1e-12) | (np.abs(dl) < 1e-12) | (np.abs(dr) < 1e-12)
    assert np.array_equal(wall, on_edge)
    assert np.allclose(np.hypot(ns.nx[wall], ns.ny[wall]), 1.0)
    # outward: the normal points away from the triangle's centroid side
    cx, cy = 0.5, -2.0 / 3.0
    assert np.all(ns.nx[wall] * (x[wall] - cx) + ns.ny[wall] * (y[wall] - cy) > 0)
    interior = ~wall
    # lattice nodes keep a clearance of 0.55 h from the slanted edges
    assert np.all(np.minimum(dl[interior], dr[interior]) >= 0.55 * h - 1e-12)
    assert abs(ns.n * h * h - 1.0) < 0.08, ns.n * h * h
    # the lid moves: u = 1 on the lid except its two corner nodes
    lid = wall & (np.abs(y) < 1e-12)
    assert np.sum(ns.u0[lid] == 1.0) == lid.sum() - 2


def test_oracle_steps_on_the_wedge_cavity():
    """Every MLS fit of the wedge is regular (no SingularStencil), and the oracle's
    first steps converge with the default normal points (longer runs need
    probes="inside", below)."""
    ns = w.wedge_cavity(33)
    fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-8)
    for _ in range(3):
        fs.step()
    assert np.all(np.isfinite(fs.u)) and np.all(np.isfinite(fs.v))
    assert np.abs(fs.u).max() <= 1.5


def test_eddy_ratios_from_the_axis_velocity_of_the_corner_mode():
    """The Moffatt post-processing (tests/eddies.py) on the exact corner mode: on
    the axis the velocity across it is r^(Re lambda - 1) cos(Im lambda ln r + phi),
    sampled at the spacing of a 401-node base (h = 1/400) over the height 2.  Its
    zeros are spaced by exp(pi / Im lambda) and its extrema fall by
    exp(pi (Re lambda - 1) / Im lambda); the resolved eddies (centres beyond 20 h)
    give both within 0.5 % (four distance and three intensity ratios)."""
    from eddies import moffatt_ratios
    g = load("moffatt_wedge.txt")
    lam = corner_eigenvalue(math.radians(g["apex_angle_deg"]))
    h = 1.0 / 400
    r = np.arange(1, 801) * h
    u = r ** (lam.real - 1) * np.cos(lam.imag * np.log(r) + 0.7)
    rr, ii = moffatt_ratios(r, u, r_min=20 * h)
    assert rr.size >= 4 and ii.size >= 3, (rr, ii)
    assert np.allclose(rr, math.exp(math.pi / lam.imag), rtol=5e-3), rr
    assert np.allclose(ii, math.exp(math.pi * (lam.real - 1) / lam.imag), rtol=5e-3), ii


def test_probes_inside_keep_the_normal_points_in_the_wedge():
    """With probes="inside" every normal point of the wedge lies in the closed
    triangle (checked against its exact edges); with the default placement the
    second points of the wall nodes next to the apex pass through the opposite
    wall.  On the square cavity the flag changes no boundary row."""
    ns = w.wedge_cavity(33, Re=100.0)
    L = math.hypot(0.5, 2.0)

    def inside(qx, qy):
        dl = (2.0 * qx - 0.5 * (-qy)) / L
        dr = (2.0 * (1.0 - qx) - 0.5 * (-qy)) / L
        return (qy <= 1e-12) & (dl >= -1e-12) & (dr >= -1e-12)

    plain = vo.Operators(ns)
    assert (~inside(*plain.probe[2])).sum() == 12
    fixed = vo.Operators(ns, probes="inside")
    for k in (1, 2):
        assert inside(*fixed.probe[k]).all(), k
    sq = w.cavity(24, Re=100.0)
    a, b = vo.Operators(sq), vo.Operators(sq, probes="inside")
    assert np.array_equal(a.probe_step, b.probe_step)
    assert (a.Nb != b.Nb).nnz == 0


def test_wedge_is_stable_only_with_the_normal_points_inside():
    """The diagnosis of the wedge's instability: with the default normal points the
    velocity grows from the apex within 100 steps (Re = 100, dt = h/4); with them
    kept inside the cavity 300 steps stay bounded by the lid speed."""
    def run(probes, steps):
        ns = w.wedge_cavity(33, Re=100.0)
        fs = vo.FractionalStep(vo.Operators(ns, probes=probes), rtol=1e-10)
        for k in range(steps):
            fs.step()
            if not np.abs(fs.u).max() < 10:
                return k + 1
        return None

    assert run("normal", 100) is not None
    assert run("inside", 300) is None

