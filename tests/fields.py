"""Helpers shared by the tests: field comparison norms and staggered positions.

Error norm (the reading used throughout): the max relative field error of a
field is max_cells |a - b| / max(max_cells |b|, floor), with floors
phi: 1, velocity: U_c, pressure: rho_L U_c^2, so that nearly-zero velocity
fields of a static case are not divided by round-off.
"""
from __future__ import annotations

import numpy as np


def max_rel_err(a, b, floor: float) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(float(np.max(np.abs(b))) if b.size else 0.0, floor)
    return float(np.max(np.abs(a - b))) / den if b.size else 0.0


def field_errors(prm: dict, a: dict, b: dict, Uc: float):
    """Per-field max relative error of state ``a`` against reference ``b``."""
    out = {}
    rhoL = prm["rhoL"]
    floors = {"phi": 1.0, "mu": 1e-3, "p": rhoL * Uc * Uc, "u": Uc, "v": Uc, "w": Uc}
    for k in ("phi", "p", "u", "v", "w", "mu"):
        if k in a and k in b and a[k] is not None and b[k] is not None:
            out[k] = max_rel_err(a[k], b[k], floors[k])
    return out


def positions(prm: dict, what: str):
    """Grid coordinates (in cells) of a field: 'c' centres, 'u','v','w' low faces.
    Returns a tuple of arrays (x, y[, z]) broadcastable to the field shape."""
    dim = prm["dim"]
    n = [prm["nx"], prm["ny"], prm["nz"]][:dim]
    axes = [np.arange(m, dtype=np.float64) + 0.5 for m in n]
    if what in ("u", "v", "w"):
        a = "uvw".index(what)
        axes[a] = axes[a] - 0.5
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return tuple(grids[::-1])
