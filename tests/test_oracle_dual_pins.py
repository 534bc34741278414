"""Pins of the oracle's dual-mesh momentum remap (sections 2.1.1 and 2.3)
against what the mathematics fixes, independently of the formulas that
compute it.  CPU only.

- The dual cells tile the plane with a quarter of each of their four cells,
  so a conservative dual remap must give every node the remapped mass
  m_p' = 1/4 (sum of the four cells' remapped masses).  The dual mass fluxes
  (quarter-box sums of primary fluxes) are chosen for exactly this; a wrong
  dual face, corner, sign or weight breaks it.
- Section 3.1's order-1 result on the primary mesh is a box formula for a
  uniform translation; "the same on the dual mesh" gives the same box formula
  for the nodal velocity, with nodes as centres.
- An order-2 limited reconstruction reproduces linear data (the limiter is
  inactive), so a uniform translation of a linear velocity field is
  remapped exactly away from the periodic seam, and a dual corner flux
  carries the exact mean of a field linear along its diagonal over the
  corner's flux region.
"""
import numpy as np
import pytest

import oracle
from paper_2208_13409_gb300 import problems as P


def _cell_mass(o, pr):
    k, r = o.get(oracle.F_K), o.get(oracle.F_RHO_MAT)
    dx = (pr.x1 - pr.x0) / pr.nx
    dy = (pr.y1 - pr.y0) / pr.ny
    return (k * r).sum(axis=0) * dx * dy


def _quarter_sums(m, periodic):
    """1/4 of the four cells around every node: wrapped (periodic) or with
    the cells mirrored across reflective walls."""
    mode = "wrap" if periodic else "symmetric"
    g = np.pad(m, 1, mode=mode)
    return 0.25 * (g[:-1, :-1] + g[:-1, 1:] + g[1:, :-1] + g[1:, 1:])


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("seed", [11, 23])
def test_nodal_mass_is_quarter_sum_of_remapped_cell_masses(periodic, seed):
    """Random three-material boxes with a diagonal drift on top of a smooth
    random flow: after each of 20 steps, m_p' = 1/4 sum m_c' at every node
    (walls: the mirrored cells complete the wall nodes' dual cells)."""
    pr = P.random_box(seed, nx=28, ny=22, nmat=3, velocity=0.25)
    pr.ux = pr.ux + 0.35
    pr.uy = pr.uy + 0.2
    if periodic:
        pr.bc = (P.BC_PERIODIC,) * 4
    o = oracle.Oracle(pr)
    for _ in range(20):
        o.step()
        mp = o.get(oracle.F_MP_NEW)
        q = _quarter_sums(_cell_mass(o, pr), periodic)
        if periodic:  # node n is node 0
            mp, q = mp[:-1, :-1], q[:-1, :-1]
        assert np.all(mp > 0.0)
        err = np.abs(mp - q).max() / q.max()
        assert err <= 1e-13, err
    # the flow actually moved mass through faces and corners
    assert np.abs(o.get(oracle.F_MC)).max() > 0.0
    assert np.abs(o.get(oracle.F_DUAL)[2:, 0]).max() > 0.0


def _translation(n, ex, ey, ulag, face_order, corner, dt=1e-2):
    """Periodic n x n box of unit density and pressure under the prescribed
    uniform displacement (ex, ey) dx per step; the dual remap carries the
    node field `ulag` = (ux, uy)."""
    pr = P.uniform(n, n, rho=1.0, p=1.0, periodic=True)
    pr.face_order, pr.corner_recon = face_order, corner
    pr.dt_fixed = dt
    dx = 1.0 / n
    o = oracle.Oracle(pr)
    vx = np.full((n + 1, n + 1), ex * dx / dt)
    vy = np.full((n + 1, n + 1), ey * dx / dt)
    o.set_prescribed(vx, vy)
    o.set_remap_velocity(*ulag)
    o.step()
    return o, dx


@pytest.mark.parametrize("sx,sy", [(1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_dual_order1_box_formula(sx, sy):
    """Section 3.1's order-1 box result on the dual mesh (nodes as centres):
    u' = u (1-ex)(1-ey) + u_{-x} ex (1-ey) + u_{-y} ey (1-ex) + u_{-x-y} ex ey,
    the shifts taken against the displacement, and m_p' = m_p."""
    n = 8
    rng = np.random.default_rng(3)
    ex, ey = 0.3, 0.2
    ux = rng.uniform(-1.0, 1.0, (n, n))
    uy = rng.uniform(-1.0, 1.0, (n, n))
    full = lambda a: np.pad(a, ((0, 1), (0, 1)), mode="wrap")
    o, dx = _translation(n, sx * ex, sy * ey, (full(ux), full(uy)), 1, P.CORNER_UPWIND)

    def box(a):
        sh = lambda di, dj: np.roll(np.roll(a, sy * dj, axis=0), sx * di, axis=1)
        return (a * (1 - ex) * (1 - ey) + sh(1, 0) * ex * (1 - ey) + sh(0, 1) * ey * (1 - ex)
                + sh(1, 1) * ex * ey)

    np.testing.assert_allclose(o.get(oracle.F_UX)[:-1, :-1], box(ux), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(o.get(oracle.F_UY)[:-1, :-1], box(uy), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(o.get(oracle.F_MP_NEW)[:-1, :-1], dx * dx, rtol=1e-13)


@pytest.mark.parametrize("axis,s", [(0, 1), (0, -1), (1, 1), (1, -1)])
def test_dual_order2_translates_linear_velocity_exactly(axis, s):
    """Order-2 dual reconstruction (Van Leer over the nodes' Lagrangian
    positions, dual width, face displacement): an axis-aligned translation of
    a velocity field linear along that axis is exact away from the seam,
    u'(x) = u(x - d)."""
    n, eps = 32, 0.3
    xn = np.arange(n + 1) / n
    X, Y = np.meshgrid(xn, xn)
    S = X if axis == 0 else Y
    ux, uy = 1.0 + 0.5 * S, 0.3 - 0.2 * S
    ex, ey = (s * eps, 0.0) if axis == 0 else (0.0, s * eps)
    o, dx = _translation(n, ex, ey, (ux, uy), 2, P.CORNER_DIAG)
    d = s * eps * dx
    inner = (slice(None), slice(4, n - 4)) if axis == 0 else (slice(4, n - 4), slice(None))
    np.testing.assert_allclose(o.get(oracle.F_UX)[inner], (1.0 + 0.5 * (S - d))[inner], rtol=1e-13)
    np.testing.assert_allclose(o.get(oracle.F_UY)[inner], (0.3 - 0.2 * (S - d))[inner], rtol=1e-13)


@pytest.mark.parametrize("sx,sy", [(1, 1), (-1, -1), (1, -1), (-1, 1)])
def test_dual_corner_carries_mean_of_diagonal_linear_field(sx, sy):
    """A translation along a diagonal (|ex| = |ey|) of a velocity field
    linear along that diagonal: every interior dual corner flux of that kind
    carries the field's exact mean over its flux region, the rectangle
    between the cell centre and the centre moved by d, taken in the
    Lagrangian configuration (the node values sit at the displaced nodes):
    u_L(c + d/2) with u_L(X) = u(X - d).  The other diagonal's corners carry
    nothing."""
    n, eps = 24, 0.25
    xn = np.arange(n + 1) / n
    X, Y = np.meshgrid(xn, xn)
    w = X + sx * sy * Y                    # coordinate along the diagonal
    ux, uy = 0.7 + 0.9 * w, -0.4 + 0.6 * w
    o, dx = _translation(n, sx * eps, sy * eps, (ux, uy), 2, P.CORNER_DIAG)
    dual = o.get(oracle.F_DUAL)
    kind = oracle.DUAL_PP if sx * sy > 0 else oracle.DUAL_PM
    other = oracle.DUAL_PM if kind == oracle.DUAL_PP else oracle.DUAL_PP
    D, PX, PY = dual[kind]
    assert np.all(dual[other] == 0.0)
    xc = (np.arange(n) + 0.5) / n
    CX, CY = np.meshgrid(xc, xc)
    d = np.array([sx, sy]) * eps * dx
    # mean over the region = value at its centroid c + d/2, in Lagrangian
    # coordinates: w(c + d/2 - d) = w(c) - (d_x + sx sy d_y)/2
    wc = CX + sx * sy * CY - 0.5 * (d[0] + sx * sy * d[1])
    inner = (slice(4, n - 4), slice(4, n - 4))
    Dm = D[:-1, :-1][inner]
    # mass flux of a corner: rho |dx dy| with the sign of the x displacement
    np.testing.assert_allclose(Dm, sx * (eps * dx) ** 2, rtol=1e-13)
    np.testing.assert_allclose((PX[:-1, :-1][inner] / Dm), (0.7 + 0.9 * wc)[inner], rtol=1e-12)
    np.testing.assert_allclose((PY[:-1, :-1][inner] / Dm), (-0.4 + 0.6 * wc)[inner], rtol=1e-12)


def test_dual_face_carries_mean_of_linear_field():
    """Dual X faces under an x translation by d: the flux through the face at
    x_f (between nodes i, i+1) is the strip [x_f, x_f + d] of the Lagrangian
    dual cell of node i, whose content is the field carried by the displaced
    nodes, u_L(X) = u(X - d); its mean is u_L(x_f + d/2) = u(x_f - d/2).  No
    Y-face or corner flux."""
    n, eps = 24, 0.3
    xn = np.arange(n + 1) / n
    X, _ = np.meshgrid(xn, xn)
    ux, uy = 2.0 - 0.7 * X, 0.5 + 0.4 * X
    o, dx = _translation(n, eps, 0.0, (ux, uy), 2, P.CORNER_DIAG)
    dual = o.get(oracle.F_DUAL)
    D, PX, PY = dual[oracle.DUAL_X]
    for kind in (oracle.DUAL_Y, oracle.DUAL_PP, oracle.DUAL_PM):
        assert np.all(dual[kind] == 0.0)
    d = eps * dx
    xf = (np.arange(n) + 0.5) / n
    xm = np.broadcast_to(xf - 0.5 * d, (n, n))
    inner = (slice(None), slice(4, n - 4))
    Dm = D[:-1, :-1]
    np.testing.assert_allclose(Dm, eps * dx * dx, rtol=1e-13)
    np.testing.assert_allclose((PX[:-1, :-1] / Dm)[inner], (2.0 - 0.7 * xm)[inner], rtol=1e-12)
    np.testing.assert_allclose((PY[:-1, :-1] / Dm)[inner], (0.5 + 0.4 * xm)[inner], rtol=1e-12)


@pytest.mark.parametrize("sx,sy", [(1, 1), (-1, -1), (1, -1), (-1, 1)])
def test_dual_fluxes_exact_under_affine_displacement(sx, sy):
    """A prescribed velocity affine in each coordinate (the nodes stretch or
    compress as well as drift, so dual widths and dual-cell centre
    displacements vary) with a carried field linear in the Lagrangian
    coordinates: an interior dual X face (between nodes i, i+1, displaced by
    d_f = mean of the two) carries u_L at the centroid of the strip between
    its Eulerian and Lagrangian positions, b0 + b1 (x_f + d_f/2); a dual
    corner carries the mean of a field linear along its diagonal over the
    rectangle between the cell centre c and c + d_c, d_c the mean of the
    cell's four node displacements (exact for a map that keeps axes)."""
    n = 24
    h = 1.0 / n
    pr = P.uniform(n, n, rho=1.0, p=1.0, periodic=False)
    pr.face_order, pr.corner_recon = 2, P.CORNER_DIAG
    xn = np.arange(n + 1) * h
    X, Y = np.meshgrid(xn, xn)
    vx = sx * 0.6 + 0.4 * (X - 0.5)
    vy = sy * 0.5 - 0.3 * (Y - 0.5)
    dt = 0.25 * h / 0.8
    pr.dt_fixed = dt
    dX, dY = dt * vx, dt * vy
    s = sx * sy
    XL, YL = X + dX, Y + dY                  # Lagrangian node positions
    ux = 0.3 + 1.7 * XL
    uy = -0.2 + 0.9 * (XL + s * YL)
    o = oracle.Oracle(pr)
    o.set_prescribed(vx, vy)
    o.set_remap_velocity(ux, uy)
    o.step()
    dual = o.get(oracle.F_DUAL)
    m = slice(4, n - 4)
    # dual X faces: (j, i) between nodes (i, j), (i+1, j)
    D, PX = dual[oracle.DUAL_X][0][:, :-1], dual[oracle.DUAL_X][1][:, :-1]
    xf = 0.5 * (X[:, :-1] + X[:, 1:])
    df = 0.5 * (dX[:, :-1] + dX[:, 1:])
    assert np.all(np.sign(D[m, m]) == sx)
    np.testing.assert_allclose((PX / D)[m, m], (0.3 + 1.7 * (xf + 0.5 * df))[m, m], rtol=1e-12)
    # dual corners at cell centres (j, i)
    kind = oracle.DUAL_PP if s > 0 else oracle.DUAL_PM
    other = oracle.DUAL_PM if s > 0 else oracle.DUAL_PP
    Dc, PYc = dual[kind][0][:-1, :-1], dual[kind][2][:-1, :-1]
    assert np.all(dual[other][0][:-1, :-1][m, m] == 0.0)
    assert np.all(np.sign(Dc[m, m]) == sx)
    cx = 0.5 * (X[:-1, :-1] + X[:-1, 1:])
    cy = 0.5 * (Y[:-1, :-1] + Y[1:, :-1])
    quad = lambda a: 0.25 * (a[:-1, :-1] + a[:-1, 1:] + a[1:, :-1] + a[1:, 1:])
    gx, gy = cx + 0.5 * quad(dX), cy + 0.5 * quad(dY)
    np.testing.assert_allclose((PYc / Dc)[m, m], (-0.2 + 0.9 * (gx + s * gy))[m, m], rtol=1e-12)
