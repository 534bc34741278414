"""Exact solution of the 1D Riemann problem for an ideal gas (both states with
the same gamma): Newton iteration on the star pressure with the standard
shock / rarefaction pressure functions, then self-similar sampling.  Used to
pin the oracle's Sod shock tube; shares nothing with the oracle."""
import math


def _fk(p, rho, pk, c, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    pr = p / pk  # rarefaction
    f = 2.0 * c / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    return f, 1.0 / (rho * c) * pr ** (-(g + 1.0) / (2.0 * g))


def star_state(rl, ul, pl, rr, ur, pr, g):
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, cl, g)
        fr, dr = _fk(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-14, p - dp)
        if abs(pn - p) < 1e-15 * p:
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(s, rl, ul, pl, rr, ur, pr, g):
    """(rho, u, p) at similarity coordinate s = (x - x0)/t."""
    ps, us = star_state(rl, ul, pl, rr, ur, pr, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    if s <= us:  # left of contact
        if ps > pl:
            sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
            if s <= sl:
                return rl, ul, pl
            return rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps
        csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
        if s <= ul - cl:
            return rl, ul, pl
        if s >= us - csl:
            return rl * (ps / pl) ** (1.0 / g), us, ps
        u = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * ul + s)
        c = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * (ul - s))
        rho = rl * (c / cl) ** (2.0 / (g - 1.0))
        return rho, u, pl * (c / cl) ** (2.0 * g / (g - 1.0))
    if ps > pr:
        sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
        if s >= sr:
            return rr, ur, pr
        return rr * (ps / pr + gm) / (gm * ps / pr + 1.0), us, ps
    csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    if s >= ur + cr:
        return rr, ur, pr
    if s <= us + csr:
        return rr * (ps / pr) ** (1.0 / g), us, ps
    u = 2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2.0 * ur + s)
    c = 2.0 / (g + 1.0) * (cr - (g - 1.0) / 2.0 * (ur - s))
    rho = rr * (c / cr) ** (2.0 / (g - 1.0))
    return rho, u, pr * (c / cr) ** (2.0 * g / (g - 1.0))
