"""Pins of the FP64 oracle against what the paper and mathematics fix
(closed forms, printed expansions, exact solutions, invariants).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2208_13409_gb300 import problems as P
import riemann_exact

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ----------------------------------------------------------------- pieces
def test_eos_matches_isentrope_derivative():
    """c^2 of the stiffened gas equals dp/drho along the isentrope de = -p dv,
    integrated numerically (section 5.2 water constants)."""
    g, pi = GOLD["water_stiffened_gas"]["gamma"], GOLD["water_stiffened_gas"]["pi_pa"]
    rho0, e0 = 1000.0, 2.2e6
    p0, c2 = oracle.eos(g, pi, rho0, e0)
    assert p0 == pytest.approx((g - 1.0) * rho0 * e0 - pi, rel=1e-15)

    def p_at(rho1, n=4000):
        # integrate de/dv = -p(rho, e) from rho0 to rho1 (RK4 in v)
        v0, v1 = 1.0 / rho0, 1.0 / rho1
        h = (v1 - v0) / n
        v, e = v0, e0
        f = lambda vv, ee: -oracle.eos(g, pi, 1.0 / vv, ee)[0]
        for _ in range(n):
            k1 = f(v, e); k2 = f(v + h / 2, e + h / 2 * k1)
            k3 = f(v + h / 2, e + h / 2 * k2); k4 = f(v + h, e + h * k3)
            e += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4); v += h
        return oracle.eos(g, pi, rho1, e)[0]

    d = 2e-5 * rho0
    num = (p_at(rho0 + d) - p_at(rho0 - d)) / (2 * d)
    assert c2 == pytest.approx(num, rel=1e-6)
    # perfect gas: textbook c^2 = gamma p / rho
    p, c2 = oracle.eos(1.4, 0.0, 1.2, 2.5)
    assert c2 == pytest.approx(1.4 * p / 1.2, rel=1e-15)


def test_cell_volume_is_shoelace_area():
    rng = np.random.default_rng(1)
    for _ in range(200):
        base = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], float) * rng.uniform(0.5, 2.0, 2)
        q = base + rng.uniform(-0.2, 0.2, (4, 2))
        ll, lr, ul, ur = q
        poly = np.array([ll, lr, ur, ul])
        x, y = poly[:, 0], poly[:, 1]
        shoelace = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
        assert oracle.cell_volume(q.ravel()) == pytest.approx(shoelace, rel=1e-13)


def test_vanleer_matches_phi_form():
    """Section 2.1.1: 1/2 (phi(r) d+ + phi(1/r) d-), r = d-/d+, phi(r) = (r+|r|)/(1+r)."""
    rng = np.random.default_rng(2)
    phi = lambda r: (r + abs(r)) / (1.0 + r)
    for _ in range(2000):
        dm, dp = rng.normal(size=2) * 10.0 ** rng.uniform(-3, 3, 2)
        r = dm / dp
        if abs(1.0 + r) < 1e-9 or abs(1.0 + 1.0 / r) < 1e-9:
            continue
        ref = 0.5 * (phi(r) * dp + phi(1.0 / r) * dm)
        assert oracle.vanleer(dm, dp) == pytest.approx(ref, rel=1e-12, abs=1e-300)
    assert oracle.vanleer(1.0, 0.0) == 0.0 and oracle.vanleer(0.0, 1.0) == 0.0
    assert oracle.vanleer(2.0, 2.0) == 2.0


def test_halfplane_area_closed_forms_and_sampling():
    rect = [(0, 0), (2, 0), (2, 1), (0, 1)]
    assert oracle.halfplane_area(rect, (1, 0), 0.5) == pytest.approx(0.5, rel=1e-15)
    assert oracle.halfplane_area(rect, (0, -1), -0.25) == pytest.approx(1.5, rel=1e-15)
    s = 1 / math.sqrt(2)
    # x + y <= 0.5: triangle of legs 0.5
    assert oracle.halfplane_area(rect, (s, s), 0.5 * s) == pytest.approx(0.125, rel=1e-14)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (400000, 2)) * [2, 1]
    for _ in range(10):
        th = rng.uniform(0, 2 * math.pi)
        n = (math.cos(th), math.sin(th))
        d = rng.uniform(-0.5, 1.5)
        mc = 2.0 * np.mean(pts @ np.array(n) <= d)
        assert oracle.halfplane_area(rect, n, d) == pytest.approx(mc, abs=6e-3)


def _rect_plic_closed_form(w, h, n, k):
    """Independent inverse of the rectangle/half-plane area (piecewise
    quadratic in the line constant)."""
    a, b = abs(n[0]) * w, abs(n[1]) * h
    if a > b:
        a, b = b, a
    lo = min(0.0, n[0] * w) + min(0.0, n[1] * h)
    if a == 0.0:
        return lo + k * b
    if k <= a / (2 * b):
        s = math.sqrt(2 * a * b * k)
    elif k <= 1 - a / (2 * b):
        s = k * b + a / 2
    else:
        s = a + b - math.sqrt(2 * a * b * (1 - k))
    return lo + s


def test_plic_places_line_by_area():
    rng = np.random.default_rng(4)
    for _ in range(300):
        w, h = rng.uniform(0.3, 3.0, 2)
        rect = [(0, 0), (w, 0), (w, h), (0, h)]
        th = rng.uniform(0, 2 * math.pi)
        n = (math.cos(th), math.sin(th))
        k = rng.uniform(1e-6, 1 - 1e-6)
        d = oracle.plic(rect, n, k * w * h)
        assert oracle.halfplane_area(rect, n, d) == pytest.approx(k * w * h, rel=1e-12, abs=1e-15)
        assert d == pytest.approx(_rect_plic_closed_form(w, h, n, k), rel=1e-10, abs=1e-12)


# ------------------------------------------------------- one-step remap pins
def _periodic_box(n, rho=1.0, p=1.0):
    pr = P.uniform(n, n, rho=rho, p=p, periodic=True)
    return pr


def _one_node(eps, n=5, centre_rho=1.0, face_order=2, corner=P.CORNER_DIAG):
    pr = _periodic_box(n)
    pr.rho[0, n // 2, n // 2] = centre_rho
    pr.face_order, pr.corner_recon = face_order, corner
    dx = (pr.x1 - pr.x0) / n
    dt = 1e-3
    pr.dt_fixed = dt
    vx = np.zeros((n + 1, n + 1)); vy = np.zeros((n + 1, n + 1))
    c = n // 2
    vx[c + 1, c + 1] = eps * dx / dt
    vy[c + 1, c + 1] = eps * dx / dt
    o = oracle.Oracle(pr)
    o.set_prescribed(vx, vy)
    o.step()
    return o, dx, c


@pytest.mark.parametrize("eps", [0.2, 0.1, 0.05, 0.02, 0.01])
def test_one_node_lagrangian_volume(eps):
    """Section 3.2: the node at the top right of the centre cell moves by
    (eps, eps) dx.  DirectCF Lagrangian volume: closed form
    1 + eps/(1+eps) + eps^2, whose expansion is the paper's 1+eps+eps^3."""
    o, dx, c = _one_node(eps)
    v = o.get(oracle.F_VOL_LAGCF)[c, c] / dx ** 2
    assert v == pytest.approx(1 + eps / (1 + eps) + eps ** 2, rel=1e-13)
    assert abs(v - (1 + eps + eps ** 3)) <= 1.5 * eps ** 4
    # neighbours that only lose volume to the centre cell
    vr = o.get(oracle.F_VOL_LAGCF)[c, c + 1] / dx ** 2
    assert vr < 1.0


@pytest.mark.parametrize("eps", [0.1, 0.05, 0.02, 0.01])
def test_one_node_corner_mass_flux(eps):
    """Section 3.2: corner mass flux / m = eps^2 - eps^3 + O(eps^4) for DirectCF;
    with upwind values it is exactly eps^2 dx^2 rho^{lagCF}/m."""
    rho_c = 2.0
    o, dx, c = _one_node(eps, centre_rho=rho_c, face_order=1, corner=P.CORNER_UPWIND)
    m = rho_c * dx * dx
    dm = o.get(oracle.F_MC)[c + 1, c + 1] / m
    vol = o.get(oracle.F_VOL_LAGCF)[c, c] / dx ** 2
    assert dm == pytest.approx(eps ** 2 / vol, rel=1e-13)
    assert abs(dm - (eps ** 2 - eps ** 3)) <= 2.0 * eps ** 4


@pytest.mark.parametrize("sx,sy", [(1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_linear_advection_order1_closed_form(sx, sy):
    """Section 3.1 boxed result (index typo read as a_{i,j-1}), for every sign
    of the velocity (the donor cells mirror accordingly)."""
    n = 8
    rng = np.random.default_rng(5)
    pr = _periodic_box(n)
    rho0 = rng.uniform(0.5, 2.0, (n, n))
    pr.rho[0] = rho0
    pr.face_order, pr.corner_recon = 1, P.CORNER_UPWIND
    dx = 1.0 / n
    ex, ey = 0.3, 0.2
    dt = 1e-2
    pr.dt_fixed = dt
    pr.ux[:] = sx * ex * dx / dt
    pr.uy[:] = sy * ey * dx / dt
    o = oracle.Oracle(pr)
    o.step()
    a = rho0
    sh = lambda di, dj: np.roll(np.roll(a, sy * dj, axis=0), sx * di, axis=1)
    ref = a * (1 - ex) * (1 - ey) + sh(1, 0) * ex * (1 - ey) + sh(0, 1) * ey * (1 - ex) + sh(1, 1) * ex * ey
    got = o.get(oracle.F_RHO_MAT)[0]
    np.testing.assert_allclose(got, ref, rtol=1e-13)
    # uniform pressure and velocity are preserved
    np.testing.assert_allclose(o.get(oracle.F_P), 1.0, rtol=1e-13)
    np.testing.assert_allclose(o.get(oracle.F_UX), sx * ex * dx / dt, rtol=1e-13)


@pytest.mark.parametrize("axis", [0, 1])
def test_order2_translates_linear_field_exactly(axis):
    """Section 2.1.1 limited linear reconstruction: on a linear field the limiter
    is inactive and an axis-aligned translation is remapped exactly (away
    from the periodic seam)."""
    n = 32
    pr = _periodic_box(n)
    dx = 1.0 / n
    xc = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc)
    s = X if axis == 0 else Y
    pr.rho[0] = 1.0 + 0.5 * s
    eps, dt = 0.3, 1e-2
    pr.dt_fixed = dt
    if axis == 0:
        pr.ux[:] = eps * dx / dt
    else:
        pr.uy[:] = eps * dx / dt
    o = oracle.Oracle(pr)
    o.step()
    got = o.get(oracle.F_RHO_MAT)[0]
    ref = 1.0 + 0.5 * (s - eps * dx)
    inner = (slice(None), slice(4, n - 4)) if axis == 0 else (slice(4, n - 4), slice(None))
    np.testing.assert_allclose(got[inner], ref[inner], rtol=1e-13)


# ------------------------------------------------------ whole-step pins
@pytest.mark.parametrize("u", [(0.0, 0.0), (0.3, -0.2), (0.5, 0.5)])
def test_uniform_state_is_preserved(u):
    pr = P.uniform(16, 12, rho=1.3, p=0.7, u=u, periodic=True)
    o = oracle.Oracle(pr)
    for _ in range(20):
        o.step()
    np.testing.assert_allclose(o.get(oracle.F_RHO), 1.3, rtol=1e-13)
    np.testing.assert_allclose(o.get(oracle.F_P), 0.7, rtol=1e-12)
    np.testing.assert_allclose(o.get(oracle.F_UX), u[0], atol=1e-13)
    np.testing.assert_allclose(o.get(oracle.F_UY), u[1], atol=1e-13)


def test_rest_state_with_walls_is_preserved():
    pr = P.uniform(10, 7, rho=0.8, p=2.0, periodic=False)
    o = oracle.Oracle(pr)
    for _ in range(10):
        o.step()
    np.testing.assert_allclose(o.get(oracle.F_P), 2.0, rtol=1e-14)
    assert np.abs(o.get(oracle.F_UX)).max() == 0.0


def test_cfl_time_step_closed_form():
    pr = P.uniform(20, 10, rho=1.1, p=0.9, u=(0.3, 0.4), periodic=True)
    o = oracle.Oracle(pr)
    dt = o.step()
    c = math.sqrt(1.4 * 0.9 / 1.1)
    h = min((pr.x1 - pr.x0) / pr.nx, (pr.y1 - pr.y0) / pr.ny)
    assert dt == pytest.approx(0.25 * h / (c + 0.5), rel=1e-14)


def test_rankine_hugoniot_matches_haas_table():
    """Input state of the shock-bubble workload against section 5.2's table."""
    g = GOLD["haas_post_shock_air"]
    rho2, p2, u2 = P.rankine_hugoniot(g["mach_of_this_build"], 1.4, 1.0, 1.0)
    c1 = math.sqrt(1.4 * g["pre_shock"]["p_pa"] / g["pre_shock"]["rho"])
    assert rho2 == pytest.approx(g["rho"], abs=2e-6)
    assert p2 == pytest.approx(g["p_pa"] / g["pre_shock"]["p_pa"], abs=1e-4)
    assert u2 / math.sqrt(1.4) == pytest.approx(g["u_m_per_s"] / c1, abs=1e-4)


def _sod_l1(nx):
    pr = P.sod(nx=nx)
    o = oracle.Oracle(pr)
    while o.t < pr.t_end:
        if o.step(pr.t_end) <= 0:
            break
    xc = (np.arange(nx) + 0.5) / nx
    ex = np.array([riemann_exact.sample((x - 0.5) / pr.t_end, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4) for x in xc])
    rho = o.get(oracle.F_RHO)[1]
    p = o.get(oracle.F_P)[1]
    ux = o.get(oracle.F_UX)[1]
    uc = 0.5 * (ux[:-1] + ux[1:])
    return (np.mean(np.abs(rho - ex[:, 0])), np.mean(np.abs(uc - ex[:, 1])), np.mean(np.abs(p - ex[:, 2])))


def test_sod_converges_to_exact_riemann_solution():
    """Whole step (Lagrange + remap + dual + CFL) against the exact solution.
    Thresholds are this build's proposal (the paper prints no Sod errors):
    first-order-in-L1 convergence through shocks and contacts."""
    e128, e256, e512 = _sod_l1(128), _sod_l1(256), _sod_l1(512)
    for q in range(3):
        order1 = math.log2(e128[q] / e256[q])
        order2 = math.log2(e256[q] / e512[q])
        lo = 0.4 if q == 1 else 0.5  # the velocity error sits in the shock offset
        assert lo <= order1 <= 1.4 and lo <= order2 <= 1.4, (q, order1, order2)
    assert e256[0] < 6e-3 and e256[1] < 1.2e-2 and e256[2] < 5e-3, e256


def test_total_energy_error_vanishes_with_dt():
    """Section 1.2: the staggered scheme conserves total energy only up to an
    O(dt^2) error per step, i.e. O(dt) at a fixed time: the relative drift
    at t = 0.2 must halve when the grid (and dt) is halved.  Mass is exact."""
    drift = []
    for nx in (128, 256, 512):
        pr = P.sod(nx=nx)
        o = oracle.Oracle(pr)
        c0 = o.get(oracle.F_CONS)
        while o.t < pr.t_end:
            if o.step(pr.t_end) <= 0:
                break
        c1 = o.get(oracle.F_CONS)
        assert abs(c1[3] - c0[3]) <= 1e-14 * c0[3]
        drift.append(abs(c1[7] - c0[7]) / c0[7])
    for a, b in zip(drift, drift[1:]):
        assert 1.6 <= a / b <= 2.4, drift


def test_sod_transpose_symmetry():
    a = oracle.Oracle(P.sod(nx=64))
    b = oracle.Oracle(P.sod(nx=64, transpose=True))
    for _ in range(40):
        a.step(); b.step()
    np.testing.assert_allclose(a.get(oracle.F_RHO), b.get(oracle.F_RHO).T, rtol=1e-12)
    np.testing.assert_allclose(a.get(oracle.F_UX), b.get(oracle.F_UY).T, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(a.get(oracle.F_K), b.get(oracle.F_K).transpose(0, 2, 1), rtol=1e-12, atol=1e-15)


def test_mirror_symmetry_shock_bubble():
    """Reduced shock-bubble, symmetric about y = 0.5: fields stay mirror
    symmetric (uy antisymmetric)."""
    pr = P.shock_bubble(nx=128, ny=32)
    o = oracle.Oracle(pr)
    for _ in range(30):
        o.step()
    r = o.get(oracle.F_RHO)
    np.testing.assert_allclose(r, r[::-1], rtol=1e-12)
    k = o.get(oracle.F_K)
    np.testing.assert_allclose(k, k[:, ::-1], atol=1e-12)
    uy = o.get(oracle.F_UY)
    np.testing.assert_allclose(uy, -uy[::-1], atol=1e-12 * np.abs(o.get(oracle.F_UX)).max())


def test_x_mirror_symmetry_random_state():
    pr = P.random_box(11, nx=24, ny=20, velocity=0.2)
    mir = pr.copy(k=pr.k[:, :, ::-1], rho=pr.rho[:, :, ::-1], p=pr.p[:, :, ::-1],
                  ux=-pr.ux[:, ::-1], uy=pr.uy[:, ::-1])
    a, b = oracle.Oracle(pr), oracle.Oracle(mir)
    for _ in range(15):
        a.step(); b.step()
    np.testing.assert_allclose(a.get(oracle.F_K), b.get(oracle.F_K)[:, :, ::-1], atol=1e-11)
    np.testing.assert_allclose(a.get(oracle.F_P), b.get(oracle.F_P)[:, ::-1], rtol=1e-10)
    np.testing.assert_allclose(a.get(oracle.F_UX), -b.get(oracle.F_UX)[:, ::-1], atol=1e-11)


@pytest.mark.parametrize("u", [(0.4, 0.0), (0.3, 0.25), (-0.2, 0.35)])
def test_translated_planar_interface_is_exact(u):
    """Axis-aligned two-material interface in uniform flow (periodic): PLIC in
    the translated rectangle is exact, so k equals the exact area fraction of
    the translated strip, and rho_a, P, u are unchanged."""
    n = 20
    pr = P.uniform(n, n, rho=1.0, p=1.0, u=u, periodic=True, nmat=2)
    xc = (np.arange(n) + 0.5) / n
    X, _ = np.meshgrid(xc, xc)
    strip = ((X > 0.3) & (X < 0.6)).astype(float)
    pr.k = np.stack([1 - strip, strip])
    pr.rho = np.stack([np.where(strip < 1, 1.0, 0.0), np.where(strip > 0, 3.0, 0.0)])
    pr.p = np.stack([np.where(strip < 1, 1.0, 0.0), np.where(strip > 0, 1.0, 0.0)])
    pr.gamma = np.array([1.4, 1.6])
    pr.pinf = np.zeros(2)
    o = oracle.Oracle(pr)
    for _ in range(12):
        o.step()
    t = o.t
    dx = 1.0 / n
    lo, hi = 0.3 + u[0] * t, 0.6 + u[0] * t
    edges = np.arange(n + 1) * dx
    frac = np.zeros(n)
    for shift in (-1.0, 0.0, 1.0):
        a = np.clip(lo + shift, edges[:-1], edges[1:])
        b = np.clip(hi + shift, edges[:-1], edges[1:])
        frac += (b - a) / dx
    k1 = o.get(oracle.F_K)[1]
    np.testing.assert_allclose(k1, np.broadcast_to(frac, (n, n)), atol=1e-12)
    rm = o.get(oracle.F_RHO_MAT)
    np.testing.assert_allclose(rm[1][k1 > 1e-9], 3.0, rtol=1e-10)
    np.testing.assert_allclose(o.get(oracle.F_P), 1.0, rtol=1e-10)
    np.testing.assert_allclose(o.get(oracle.F_UX), u[0], atol=1e-12)


def test_diagonal_planar_interface_is_exact():
    """45-degree interface: Youngs' 9-point gradient gives the exact normal, so
    the translated half-plane is reproduced to round-off."""
    n = 24
    pr = P.uniform(n, n, rho=1.0, p=1.0, u=(0.3, 0.3), periodic=False, nmat=2)
    dx = 1.0 / n
    # exact fraction of {x + y < 1} in each cell
    I, J = np.meshgrid(np.arange(n), np.arange(n))
    s = I + J  # cell spans x+y in [s, s+2] dx
    f = np.where(s + 2 <= n, 1.0, np.where(s >= n, 0.0, 0.0))
    diag = (s + 1 == n)
    f[diag] = 0.5
    pr.k = np.stack([f, 1 - f])
    pr.rho = np.stack([np.where(f > 0, 1.0, 0), np.where(f < 1, 2.0, 0)])
    pr.p = np.stack([np.where(f > 0, 1.0, 0), np.where(f < 1, 1.0, 0)])
    pr.gamma = np.array([1.4, 1.4]); pr.pinf = np.zeros(2)
    # prescribed uniform velocity, fixed dt, single step
    pr.dt_fixed = 0.2 * dx / 0.3
    o = oracle.Oracle(pr)
    vx = np.full((n + 1, n + 1), 0.3)
    o.set_prescribed(vx, vx)
    o.step()
    shift = 2 * 0.3 * pr.dt_fixed  # the line x + y = 1 moves to x + y = 1 + shift
    kk = o.get(oracle.F_K)[0]
    checked = 0
    for j in range(3, n - 3):
        for i in range(3, n - 3):
            c = 1 + shift - (i + j) * dx  # cell-local u + v < c, u, v in [0, dx]
            if c <= 0:
                ex = 0.0
            elif c >= 2 * dx:
                ex = 1.0
            elif c <= dx:
                ex = 0.5 * c * c / dx ** 2
            else:
                ex = 1 - 0.5 * (2 * dx - c) ** 2 / dx ** 2
            checked += 0.0 < ex < 1.0
            assert kk[j, i] == pytest.approx(ex, abs=1e-12), (i, j)
    assert checked >= 10


def test_conservation_multimaterial_periodic():
    """Mass per material, total mass, momentum (periodic) to round-off; internal
    energy changes only through the Lagrange work."""
    pr = P.random_box(7, nx=32, ny=28, nmat=3, velocity=0.3)
    pr.bc = (P.BC_PERIODIC,) * 4
    o = oracle.Oracle(pr)
    c0 = o.get(oracle.F_CONS)
    for _ in range(25):
        o.step()
    c1 = o.get(oracle.F_CONS)
    for a in range(3):
        assert c1[a] == pytest.approx(c0[a], rel=1e-12)
    assert c1[3] == pytest.approx(c0[3], rel=1e-13)
    scale = c0[3] * 0.3
    assert abs(c1[4] - c0[4]) <= 1e-12 * scale and abs(c1[5] - c0[5]) <= 1e-12 * scale


def test_volume_fractions_bounded_three_materials():
    pr = P.triple_point(nx=70, ny=30)
    o = oracle.Oracle(pr)
    for _ in range(60):
        o.step()
        k = o.get(oracle.F_K)
        assert k.min() >= 0.0 and k.max() <= 1.0
        assert np.abs(k.sum(axis=0) - 1.0).max() <= 1e-14
    assert ((k > 0).sum(axis=0) == 3).any(), "expected cells holding all three materials"


def test_cells_and_edge_sizes():
    """Smallest grids and both boundary kinds run and keep invariants."""
    for nx, ny in [(2, 2), (2, 3), (3, 5)]:
        for per in (True, False):
            pr = P.random_box(3, nx=nx, ny=ny, velocity=0.1)
            if per:
                pr.bc = (P.BC_PERIODIC,) * 4
            o = oracle.Oracle(pr)
            for _ in range(5):
                o.step()
            k = o.get(oracle.F_K)
            assert np.abs(k.sum(axis=0) - 1).max() <= 1e-14
    # t_end reached: no step taken
    o = oracle.Oracle(P.sod(nx=16))
    assert o.step(0.0) == 0.0


# ------------------------------------------ comparator remaps (section 2)
def _one_node_remap(eps, remap, centre_rho):
    """Mono-material one-node displacement (section 3.2) with upwind values
    (the order-1 remap is linear in rho, so the centre's excess density can
    be isolated by subtracting the uniform run)."""
    n = 5
    pr = _periodic_box(n)
    pr.rho[0, n // 2, n // 2] = centre_rho
    pr.face_order, pr.corner_recon, pr.remap = 1, P.CORNER_UPWIND, remap
    dx = 1.0 / n
    dt = 1e-3
    pr.dt_fixed = dt
    vx = np.zeros((n + 1, n + 1)); vy = np.zeros((n + 1, n + 1))
    c = n // 2
    vx[c + 1, c + 1] = eps * dx / dt
    vy[c + 1, c + 1] = eps * dx / dt
    o = oracle.Oracle(pr)
    o.set_prescribed(vx, vy)
    o.step()
    return o.get(oracle.F_RHO_MAT)[0], c


@pytest.mark.parametrize("eps", [0.2, 0.1, 0.05, 0.01])
def test_one_node_lagrangian_volume_ad_and_direct(eps):
    """Section 3.2: the centre's effective Lagrangian volume m^n / m^{proj} is
    (1 + eps/2)^2 = 1 + eps + eps^2/4 for AD (two sweeps, each adding half
    of the displaced node's area) and exactly 1 + eps for Direct."""
    for remap, ref in ((P.REMAP_AD, (1 + eps / 2) ** 2), (P.REMAP_DIRECT, 1 + eps)):
        r2, c = _one_node_remap(eps, remap, 3.0)
        r1, _ = _one_node_remap(eps, remap, 1.0)
        kept = (r2[c, c] - r1[c, c]) / 2.0        # excess mass left in the centre / excess mass
        assert 1.0 / kept == pytest.approx(ref, rel=1e-13), remap


@pytest.mark.parametrize("eps", [0.1, 0.05, 0.02, 0.01])
def test_one_node_corner_mass_ad_and_direct(eps):
    """Section 3.2: mass reaching the diagonal cell through the top-right
    corner, per unit of the centre's mass.  Direct: 0.  AD (X then Y,
    eps' = 0): (eps^2/4)/(1+eps/2)^2, whose expansion is the paper's
    eps^2/4 - eps^3/4."""
    r2, c = _one_node_remap(eps, P.REMAP_DIRECT, 3.0)
    r1, _ = _one_node_remap(eps, P.REMAP_DIRECT, 1.0)
    assert abs(r2[c + 1, c + 1] - r1[c + 1, c + 1]) <= 1e-14
    r2, c = _one_node_remap(eps, P.REMAP_AD, 3.0)
    r1, _ = _one_node_remap(eps, P.REMAP_AD, 1.0)
    dm = (r2[c + 1, c + 1] - r1[c + 1, c + 1]) / 2.0
    assert dm == pytest.approx((eps ** 2 / 4) / (1 + eps / 2) ** 2, rel=1e-12)
    assert abs(dm - (eps ** 2 / 4 - eps ** 3 / 4)) <= eps ** 4


@pytest.mark.parametrize("remap", [1, 2])
@pytest.mark.parametrize("sx,sy", [(1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_linear_advection_order1_ad_and_direct(remap, sx, sy):
    """Section 3.1: uniform translation at order 1.  AD reproduces the
    boxed nine-point formula (the same as DirectCF); Direct is the
    five-point a (1 - ex - ey) + a_{i-1,j} ex + a_{i,j-1} ey."""
    n = 8
    rng = np.random.default_rng(6)
    pr = _periodic_box(n)
    rho0 = rng.uniform(0.5, 2.0, (n, n))
    pr.rho[0] = rho0
    pr.face_order, pr.corner_recon, pr.remap = 1, P.CORNER_UPWIND, remap
    dx = 1.0 / n
    ex, ey = 0.3, 0.2
    dt = 1e-2
    pr.dt_fixed = dt
    pr.ux[:] = sx * ex * dx / dt
    pr.uy[:] = sy * ey * dx / dt
    o = oracle.Oracle(pr)
    o.step()
    a = rho0
    sh = lambda di, dj: np.roll(np.roll(a, sy * dj, axis=0), sx * di, axis=1)
    if remap == P.REMAP_AD:
        ref = a * (1 - ex) * (1 - ey) + sh(1, 0) * ex * (1 - ey) + sh(0, 1) * ey * (1 - ex) + sh(1, 1) * ex * ey
    else:
        ref = a * (1 - ex - ey) + sh(1, 0) * ex + sh(0, 1) * ey
    np.testing.assert_allclose(o.get(oracle.F_RHO_MAT)[0], ref, rtol=1e-13)
    np.testing.assert_allclose(o.get(oracle.F_UX), sx * ex * dx / dt, rtol=1e-13)
    if remap == P.REMAP_AD:  # the second step sweeps Y first: same result for uniform flow
        o.step()
        a = ref
        ref2 = a * (1 - ex) * (1 - ey) + sh(1, 0) * ex * (1 - ey) + sh(0, 1) * ey * (1 - ex) + sh(1, 1) * ex * ey
        np.testing.assert_allclose(o.get(oracle.F_RHO_MAT)[0], ref2, rtol=1e-13)


@pytest.mark.parametrize("remap", [1, 2])
def test_comparator_remaps_preserve_uniform_state_and_conserve(remap):
    pr = P.uniform(16, 12, rho=1.3, p=0.7, u=(0.3, -0.2), periodic=True).copy(remap=remap)
    o = oracle.Oracle(pr)
    for _ in range(12):
        o.step()
    np.testing.assert_allclose(o.get(oracle.F_RHO), 1.3, rtol=1e-13)
    np.testing.assert_allclose(o.get(oracle.F_P), 0.7, rtol=1e-12)
    np.testing.assert_allclose(o.get(oracle.F_UX), 0.3, rtol=1e-13)
    pr = P.random_box(7, nx=32, ny=28, nmat=3, velocity=0.3).copy(remap=remap, bc=(P.BC_PERIODIC,) * 4)
    o = oracle.Oracle(pr)
    c0 = o.get(oracle.F_CONS)
    for _ in range(20):
        o.step()
        k = o.get(oracle.F_K)
        assert k.min() >= 0.0 and np.abs(k.sum(axis=0) - 1.0).max() <= 1e-14
    c1 = o.get(oracle.F_CONS)
    for a in range(4):
        assert c1[a] == pytest.approx(c0[a], rel=1e-12)
    scale = c0[3] * 0.3
    assert abs(c1[4] - c0[4]) <= 1e-12 * scale and abs(c1[5] - c0[5]) <= 1e-12 * scale


def test_ad_translates_axis_aligned_interface_exactly():
    """AD multi-material (section 4.3): a vertical interface moving along x
    is remapped exactly by the X sweep; the Y sweep has nothing to do."""
    n = 16
    pr = P.uniform(n, n, rho=1.0, p=1.0, u=(0.0, 0.0), periodic=True, nmat=2).copy(remap=P.REMAP_AD)
    x = (np.arange(n) + 0.5) / n
    ka = np.where(x < 0.5, 1.0, 0.0)[None, :].repeat(n, axis=0)
    pr.k = np.stack([ka, 1.0 - ka])
    pr.rho = np.stack([np.where(ka > 0, 1.0, 0.0), np.where(ka < 1, 1.0, 0.0)])
    pr.p = np.stack([np.where(ka > 0, 1.0, 0.0), np.where(ka < 1, 1.0, 0.0)])
    eps, dt = 0.25, 1e-2
    pr.dt_fixed = dt
    pr.ux[:] = eps / n / dt
    o = oracle.Oracle(pr)
    o.step()
    k = o.get(oracle.F_K)[0]
    col = np.zeros(n)
    col[:8] = 1.0
    col[8] = eps
    col[0] = 1.0 - eps   # the periodic image of the interface at x = 0
    np.testing.assert_allclose(k, col[None, :].repeat(n, axis=0), atol=1e-14)


# --------------------------------------------- corner reconstructions (3.3)
def _linear_translation(corner, rho_of, ex=0.2, ey=0.1, n=12):
    """Uniform translation of a linear density field (uniform p and u, so
    rho^{lagCF} = rho and every Lagrangian rectangle is the Eulerian cell
    shifted by (ex dx, ey dy))."""
    pr = _periodic_box(n)
    I, J = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    pr.rho[0] = rho_of(I, J)
    pr.corner_recon = corner
    dx = 1.0 / n
    dt = 1e-2
    pr.dt_fixed = dt
    pr.ux[:] = ex * dx / dt
    pr.uy[:] = ey * dx / dt
    o = oracle.Oracle(pr)
    o.step()
    return o, dx, pr.rho[0]


def test_corner_average_is_clamped_to_the_donor():
    """Average corner value 1/2 (a_donor + a_receiver), clamped to a_donor."""
    for rho_of, clamps in ((lambda I, J: 2.0 - 0.05 * I - 0.03 * J, False), (lambda I, J: 1.0 + 0.05 * I + 0.03 * J, True)):
        o, dx, rho = _linear_translation(P.CORNER_AVG, rho_of)
        rc, rr = rho[5, 5], rho[6, 6]
        rp = rc if clamps else 0.5 * (rc + rr)
        assert o.get(oracle.F_MC)[6, 6] == pytest.approx(rp * 0.2 * dx * 0.1 * dx, rel=1e-13)


def test_corner_xy_formula():
    """x-y corner value a_c + delta_x/2 (dx^{lag} - dt u_x) + delta_y/2 (dy^{lag} - dt u_y)
    with exact slopes on a linear field."""
    o, dx, rho = _linear_translation(P.CORNER_XY, lambda I, J: 1.0 + 0.05 * I + 0.03 * J)
    rp = rho[5, 5] + 0.5 * 0.05 * (1 - 0.2) + 0.5 * 0.03 * (1 - 0.1)
    assert o.get(oracle.F_MC)[6, 6] == pytest.approx(rp * 0.2 * dx * 0.1 * dx, rel=1e-13)


def test_multidimensional_reconstruction_limited_plane():
    """Least-squares plane: G is the exact gradient of a linear field, scaled
    to the norm min(|d_x|, |d_y|, |d_v|, |d_vperp|) of the limited 1D slopes,
    evaluated at the flux region's centroid (corner and face)."""
    o, dx, rho = _linear_translation(P.CORNER_LSQ, lambda I, J: 1.0 + 0.05 * I + 0.03 * J)
    b, c = 0.05 / dx, 0.03 / dx
    m = min(abs(b), abs(c), abs(b + c) / math.sqrt(2), abs(b - c) / math.sqrt(2))
    phi = m / math.hypot(b, c)
    # corner (donor (5,5)): region [1, 1.2] x [1, 1.1] dx, Lagrangian centre (0.7, 0.6) dx
    rp = rho[5, 5] + phi * (b * 0.4 * dx + c * 0.45 * dx)
    assert o.get(oracle.F_MC)[6, 6] == pytest.approx(rp * 0.2 * dx * 0.1 * dx, rel=1e-13)
    # X face between (5,5) and (6,5): region [1, 1.2] x [0.1, 1] dx (trapezoid rows)
    rf = rho[5, 5] + phi * (b * 0.4 * dx - c * 0.05 * dx)
    assert o.get(oracle.F_MX)[5, 6] == pytest.approx(rf * 0.2 * dx * 0.9 * dx, rel=1e-13)
    # an axis-aligned gradient has a zero limited slope across it: order 1
    o, dx, rho = _linear_translation(P.CORNER_LSQ, lambda I, J: 1.0 + 0.05 * I)
    assert o.get(oracle.F_MX)[5, 6] == pytest.approx(rho[5, 5] * 0.2 * dx * 0.9 * dx, rel=1e-13)


@pytest.mark.parametrize("corner", [2, 3, 4])
def test_corner_variants_conserve_and_stay_bounded(corner):
    pr = P.random_box(9, nx=30, ny=26, nmat=3, velocity=0.3).copy(corner_recon=corner, bc=(P.BC_PERIODIC,) * 4)
    o = oracle.Oracle(pr)
    c0 = o.get(oracle.F_CONS)
    for _ in range(20):
        o.step()
        k = o.get(oracle.F_K)
        assert k.min() >= 0.0 and np.abs(k.sum(axis=0) - 1.0).max() <= 1e-14
    c1 = o.get(oracle.F_CONS)
    for a in range(4):
        assert c1[a] == pytest.approx(c0[a], rel=1e-12)
