"""Comparison helpers for GPU-vs-oracle parity.

Per-material fields are compared in extensive form (k, k rho, k rho e):
the intensive rho_a, e_a of a material that is almost absent from a cell
are a difference of nearly equal numbers divided by a tiny volume, so their
relative value is ill-conditioned at any precision.  Mixture fields are
compared directly; the node velocity is compared as one vector field
against the largest speed component (a component that vanishes in exact
arithmetic, like u_y of a 1D problem, has no meaningful relative error)."""
import numpy as np

import oracle
from paper_2208_13409_gb300 import lr


def fields(obj, mod):
    k = obj.get(mod.F_K)
    r = obj.get(mod.F_RHO_MAT)
    e = obj.get(mod.F_E_MAT)
    return {"k": k, "k_rho": k * r, "k_rho_e": k * r * e,
            "rho": obj.get(mod.F_RHO), "p": obj.get(mod.F_P),
            "u": np.stack([obj.get(mod.F_UX), obj.get(mod.F_UY)])}


def max_rel(g, o):
    """max |g - o| / max |o| (relative to the field's range)."""
    scale = np.abs(o).max()
    if scale == 0.0:
        return float(np.abs(g).max())
    return float(np.abs(g - o).max() / scale)


def l1_rel(g, o):
    """sum |g - o| / sum |o|."""
    s = np.abs(o).sum()
    if s == 0.0:
        return float(np.abs(g).sum())
    return float(np.abs(g - o).sum() / s)


def compare(sim, orc, metric=max_rel):
    fg, fo = fields(sim, lr), fields(orc, oracle)
    return {key: metric(fg[key], fo[key]) for key in fo}
