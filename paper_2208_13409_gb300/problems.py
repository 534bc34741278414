"""Seeded synthetic initial states for the Lagrange-Remap step.

This module holds no arithmetic of the scheme itself: it only builds initial
states (volume fractions, material densities and pressures, node
velocities) and their configuration.  Both the oracle tests and the CUDA
path consume the same arrays, so the two never share method code.

Workloads (sizes from the workload list of this project):
  * two-material Sod tube, 256 x 4 on [0,1] x [0,1/64] (section 5 style set-up)
  * three-material triple point, 1400 x 600 on [0,7] x [0,3]
  * shock-bubble, 4096 x 1024 on [0,4] x [0,1], Mach 1.22 air shock on a
    helium disc (the HAAS set-up of section 5.2, rescaled)
  * random multi-material boxes (ensemble members), seeded
  * air/water serving requests (stiffened-gas water, section 5.2)
Arrays: cells [nmat][ny][nx] (x fastest), nodes [ny+1][nx+1].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

BC_REFLECT, BC_PERIODIC = 0, 1
CORNER_UPWIND, CORNER_DIAG, CORNER_AVG, CORNER_XY, CORNER_LSQ = 0, 1, 2, 3, 4
REMAP_DIRECTCF, REMAP_DIRECT, REMAP_AD = 0, 1, 2


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    gamma: np.ndarray          # [nmat]
    pinf: np.ndarray           # [nmat] stiffened-gas constant pi of p=(g-1)rho e - pi
    k: np.ndarray              # [nmat][ny][nx]
    rho: np.ndarray            # [nmat][ny][nx]
    p: np.ndarray              # [nmat][ny][nx]
    ux: np.ndarray             # [ny+1][nx+1]
    uy: np.ndarray             # [ny+1][nx+1]
    bc: Sequence[int] = (BC_REFLECT,) * 4
    cfl: float = 0.25
    a1: float = 0.5
    a2: float = 1.0
    face_order: int = 2
    corner_recon: int = CORNER_DIAG
    dt_fixed: float = 0.0
    t_end: float = 1e300
    remap: int = 0                 # REMAP_DIRECTCF, REMAP_DIRECT or REMAP_AD

    @property
    def nmat(self) -> int:
        return int(self.gamma.shape[0])

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def copy(self, **kw) -> "Problem":
        d = {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}
        for key in ("gamma", "pinf", "k", "rho", "p", "ux", "uy"):
            d[key] = np.array(d[key], dtype=np.float64, copy=True)
        d.update(kw)
        return Problem(**d)


def _centres(nx, ny, x0, x1, y0, y1):
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * dx
    yc = y0 + (np.arange(ny) + 0.5) * dy
    return np.meshgrid(xc, yc)  # [ny][nx]


def _nodes(nx, ny, x0, x1, y0, y1):
    xn = x0 + np.arange(nx + 1) * (x1 - x0) / nx
    yn = y0 + np.arange(ny + 1) * (y1 - y0) / ny
    return np.meshgrid(xn, yn)


def disc_fraction(nx, ny, x0, x1, y0, y1, cx, cy, r, sub=8) -> np.ndarray:
    """Fraction of each cell inside the disc, by sub x sub point sampling
    (computed once on the host and handed to both implementations)."""
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    out = np.zeros((ny, nx))
    i0 = max(0, int(math.floor((cx - r - x0) / dx)) - 1)
    i1 = min(nx, int(math.ceil((cx + r - x0) / dx)) + 1)
    j0 = max(0, int(math.floor((cy - r - y0) / dy)) - 1)
    j1 = min(ny, int(math.ceil((cy + r - y0) / dy)) + 1)
    if i1 <= i0 or j1 <= j0:
        return out
    off = (np.arange(sub) + 0.5) / sub
    xs = x0 + (np.arange(i0, i1)[:, None] + off[None, :]) * dx          # [ni][sub]
    ys = y0 + (np.arange(j0, j1)[:, None] + off[None, :]) * dy          # [nj][sub]
    dx2 = (xs - cx) ** 2
    dy2 = (ys - cy) ** 2
    inside = (dy2[:, None, :, None] + dx2[None, :, None, :]) <= r * r  # [nj][ni][sub][sub]
    out[j0:j1, i0:i1] = inside.mean(axis=(2, 3))
    return out


def rankine_hugoniot(mach: float, gamma: float, rho1: float, p1: float):
    """Post-shock (rho2, p2, u2) of a shock of Mach number `mach` running into
    gas at rest (textbook normal-shock relations)."""
    g = gamma
    m2 = mach * mach
    rho2 = rho1 * (g + 1.0) * m2 / ((g - 1.0) * m2 + 2.0)
    p2 = p1 * (2.0 * g * m2 - (g - 1.0)) / (g + 1.0)
    c1 = math.sqrt(g * p1 / rho1)
    u2 = c1 * 2.0 / (g + 1.0) * (mach - 1.0 / mach)
    return rho2, p2, u2


def _zeros_nodes(nx, ny):
    return np.zeros((ny + 1, nx + 1)), np.zeros((ny + 1, nx + 1))


def sod(nx: int = 256, ny: int = 4, transpose: bool = False) -> Problem:
    """Two-material Sod tube: A (rho 1, p 1) for x<0.5, B (0.125, 0.1),
    gamma 1.4 both, walls, run to t = 0.2.  `transpose` swaps the axes."""
    if transpose:
        nx, ny = ny, nx
        x0, x1, y0, y1 = 0.0, 1.0 / 64.0, 0.0, 1.0
        _, s = _centres(nx, ny, x0, x1, y0, y1)
    else:
        x0, x1, y0, y1 = 0.0, 1.0, 0.0, 1.0 / 64.0
        s, _ = _centres(nx, ny, x0, x1, y0, y1)
    left = (s < 0.5).astype(np.float64)
    k = np.stack([left, 1.0 - left])
    rho = np.stack([np.where(left > 0, 1.0, 0.0), np.where(left > 0, 0.0, 0.125)])
    p = np.stack([np.where(left > 0, 1.0, 0.0), np.where(left > 0, 0.0, 0.1)])
    ux, uy = _zeros_nodes(nx, ny)
    return Problem("sod", nx, ny, x0, x1, y0, y1, np.array([1.4, 1.4]), np.zeros(2),
                   k, rho, p, ux, uy, t_end=0.2)


def triple_point(nx: int = 1400, ny: int = 600) -> Problem:
    """Three-material triple point on [0,7] x [0,3]: x<1 (1, 1, gamma 1.5);
    x>1, y<1.5 (1, 0.1, gamma 1.4); x>1, y>1.5 (0.125, 0.1, gamma 1.5);
    at rest, walls, run to t = 5."""
    x0, x1, y0, y1 = 0.0, 7.0, 0.0, 3.0
    xc, yc = _centres(nx, ny, x0, x1, y0, y1)
    m0 = (xc < 1.0).astype(np.float64)
    m1 = ((xc > 1.0) & (yc < 1.5)).astype(np.float64)
    m2 = 1.0 - m0 - m1
    k = np.stack([m0, m1, m2])
    rho = np.stack([m0 * 1.0, m1 * 1.0, m2 * 0.125])
    p = np.stack([m0 * 1.0, m1 * 0.1, m2 * 0.1])
    ux, uy = _zeros_nodes(nx, ny)
    return Problem("triple_point", nx, ny, x0, x1, y0, y1, np.array([1.5, 1.4, 1.5]), np.zeros(3),
                   k, rho, p, ux, uy, t_end=5.0)


def shock_bubble(nx: int = 4096, ny: int = 1024, x_shock: float = 0.6, mach: float = 1.22) -> Problem:
    """Air (gamma 1.4, rho 1, p 1) with a Mach 1.22 shock at x = x_shock moving
    right (post-shock Rankine-Hugoniot state behind it) and a helium disc
    (gamma 1.648, rho 0.138, p 1) of radius 0.25 centred at (1, 0.5); walls."""
    x0, x1, y0, y1 = 0.0, 4.0, 0.0, 1.0
    xc, _ = _centres(nx, ny, x0, x1, y0, y1)
    kb = disc_fraction(nx, ny, x0, x1, y0, y1, 1.0, 0.5, 0.25)
    ka = 1.0 - kb
    rho2, p2, u2 = rankine_hugoniot(mach, 1.4, 1.0, 1.0)
    post = xc < x_shock
    rho_a = np.where(post, rho2, 1.0)
    p_a = np.where(post, p2, 1.0)
    k = np.stack([ka, kb])
    rho = np.stack([np.where(ka > 0, rho_a, 0.0), np.where(kb > 0, 0.138, 0.0)])
    p = np.stack([np.where(ka > 0, p_a, 0.0), np.where(kb > 0, 1.0, 0.0)])
    xn, _ = _nodes(nx, ny, x0, x1, y0, y1)
    ux = np.where(xn < x_shock, u2, 0.0)
    uy = np.zeros_like(ux)
    return Problem("shock_bubble", nx, ny, x0, x1, y0, y1, np.array([1.4, 1.648]), np.zeros(2),
                   k, rho, p, ux, uy)


def uniform(nx: int, ny: int, rho: float = 1.0, p: float = 1.0, u=(0.0, 0.0),
            periodic: bool = True, gamma: float = 1.4, nmat: int = 1, k=None) -> Problem:
    """Uniform state; with nmat > 1 the volume fractions `k` (a [nmat] vector,
    or arrays) describe identical materials."""
    x0, x1, y0, y1 = 0.0, 1.0, 0.0, 1.0 * ny / nx
    if k is None:
        k = np.zeros((nmat, ny, nx))
        k[0] = 1.0
    kk = np.asarray(k, dtype=np.float64)
    if kk.ndim == 1:
        kk = np.broadcast_to(kk[:, None, None], (nmat, ny, nx)).copy()
    rr = np.where(kk > 0, rho, 0.0)
    pp = np.where(kk > 0, p, 0.0)
    ux = np.full((ny + 1, nx + 1), float(u[0]))
    uy = np.full((ny + 1, nx + 1), float(u[1]))
    bc = (BC_PERIODIC,) * 4 if periodic else (BC_REFLECT,) * 4
    return Problem("uniform", nx, ny, x0, x1, y0, y1, np.full(nmat, gamma), np.zeros(nmat),
                   kk, rr, pp, ux, uy, bc=bc)


def random_box(seed: int, nx: int = None, ny: int = None, nmat: int = None,
               sides: Sequence[int] = (64, 96, 128, 192, 256, 384, 512),
               velocity: float = 0.0) -> Problem:
    """One ensemble member: square grid from `sides`, 1-3 random axis-aligned
    rectangles or discs of other materials in a background material, gamma in
    [1.3, 1.7], rho log-uniform in [0.1, 10], p log-uniform in [0.01, 10],
    walls, zero velocity (or a random smooth field when `velocity` > 0)."""
    rng = np.random.default_rng(seed)
    side = int(rng.choice(sides))
    nx = nx or side
    ny = ny or side
    nreg = int(rng.integers(1, 4))
    M = nmat or min(3, 1 + nreg)
    x0, x1, y0, y1 = 0.0, 1.0, 0.0, float(ny) / nx
    xc, yc = _centres(nx, ny, x0, x1, y0, y1)
    k = np.zeros((M, ny, nx))
    k[0] = 1.0
    for q in range(nreg):
        a = 1 + (q % (M - 1)) if M > 1 else 0
        if a == 0:
            continue
        if rng.random() < 0.5:
            cx, cy = rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8) * y1
            r = rng.uniform(0.05, 0.2) * min(1.0, y1)
            f = disc_fraction(nx, ny, x0, x1, y0, y1, cx, cy, r)
        else:
            xa, xb = np.sort(rng.uniform(0.1, 0.9, 2))
            ya, yb = np.sort(rng.uniform(0.1, 0.9, 2)) * y1
            f = ((xc > xa) & (xc < xb) & (yc > ya) & (yc < yb)).astype(np.float64)
        k = (1.0 - f)[None] * k
        k[a] += f
    k = np.clip(k, 0.0, 1.0)
    k /= k.sum(axis=0, keepdims=True)
    gam = rng.uniform(1.3, 1.7, M)
    rho = np.exp(rng.uniform(math.log(0.1), math.log(10.0), M))
    pr = np.exp(rng.uniform(math.log(0.01), math.log(10.0), M))
    R = np.where(k > 0, rho[:, None, None], 0.0)
    P = np.where(k > 0, pr[:, None, None], 0.0)
    ux, uy = _zeros_nodes(nx, ny)
    if velocity > 0.0:
        xn, yn = _nodes(nx, ny, x0, x1, y0, y1)
        ph = rng.uniform(0, 2 * math.pi, 2)
        ux = velocity * np.sin(2 * math.pi * xn + ph[0]) * np.cos(2 * math.pi * yn)
        uy = velocity * np.cos(2 * math.pi * xn) * np.sin(2 * math.pi * yn + ph[1])
    return Problem(f"random_box{seed}", nx, ny, x0, x1, y0, y1, gam, np.zeros(M),
                   k, R, P, ux, uy)


def ensemble(n: int = 512, seed: int = 2208) -> List[Problem]:
    """The batched ensemble: member i uses seed + i."""
    return [random_box(seed + i) for i in range(n)]


def air_water(seed: int, side: int = None, steps_range=(200, 2000), sub: int = 8) -> Problem:
    """One serving request on [0,1]^2 m: air (gamma 1.4, rho 1.2, p 1e5) and
    stiffened-gas water (gamma 4.4, p_inf 6e8 Pa so pi = gamma p_inf,
    rho 1000, p 1e5) as a water column (x in [0.4,0.6]) or a droplet, hit by
    an air shock from the left (pressure ratio log-uniform in [10,100]) at
    x = 0.1.  The requested step count is stored as attribute `steps`; `sub`
    is the droplet's sampling per cell side for the volume fractions."""
    rng = np.random.default_rng(seed)
    if side is None:
        side = int(round(math.exp(rng.uniform(math.log(128), math.log(2048)))))
    nx = ny = side
    x0, x1, y0, y1 = 0.0, 1.0, 0.0, 1.0
    xc, yc = _centres(nx, ny, x0, x1, y0, y1)
    if rng.random() < 0.5:
        kw = ((xc > 0.4) & (xc < 0.6)).astype(np.float64)
    else:
        kw = disc_fraction(nx, ny, x0, x1, y0, y1, 0.5, 0.5, rng.uniform(0.05, 0.2), sub=sub)
    ka = 1.0 - kw
    ratio = math.exp(rng.uniform(math.log(10.0), math.log(100.0)))
    g = 1.4
    # shock Mach number giving pressure ratio `ratio` (normal-shock relation)
    mach = math.sqrt(((g + 1.0) * ratio + (g - 1.0)) / (2.0 * g))
    rho2, p2, u2 = rankine_hugoniot(mach, g, 1.2, 1e5)
    post = xc < 0.1
    k = np.stack([ka, kw])
    rho = np.stack([np.where(ka > 0, np.where(post, rho2, 1.2), 0.0), np.where(kw > 0, 1000.0, 0.0)])
    p = np.stack([np.where(ka > 0, np.where(post, p2, 1e5), 0.0), np.where(kw > 0, 1e5, 0.0)])
    xn, _ = _nodes(nx, ny, x0, x1, y0, y1)
    ux = np.where(xn < 0.1, u2, 0.0)
    uy = np.zeros_like(ux)
    prob = Problem(f"air_water{seed}", nx, ny, x0, x1, y0, y1, np.array([1.4, 4.4]),
                   np.array([0.0, 4.4 * 6e8]), k, rho, p, ux, uy)
    prob.steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
    return prob
