"""The interface position of the capillary wave at its symmetry plane y = 0,
from a phase field on the cell centres (shared by the capillary-wave tests)."""
from __future__ import annotations

import numpy as np


def row_crossing(phi_row, dx, W):
    """x of the phi = 0 crossing of one row (cell centres at (i + 1/2) dx): each
    of the two cells around the sign change gives it through the inverse of
    the equilibrium profile tanh(2 d / W), and the two are averaged."""
    s = np.nonzero((phi_row[:-1] < 0.0) & (phi_row[1:] >= 0.0))[0]
    i = int(s[0])
    a, b = np.clip(phi_row[i], -0.999999, 0.999999), np.clip(phi_row[i + 1], -0.999999, 0.999999)
    xa = (i + 0.5) * dx - 0.5 * W * np.arctanh(a)
    xb = (i + 1.5) * dx - 0.5 * W * np.arctanh(b)
    return 0.5 * (xa + xb)


def h_tilde(phi, prm):
    """(h_eq - h_0) / A_p with h_0 the interface position at y = 0: the rows at
    y = dx/2 and 3 dx/2 extrapolated with the even profile h = a + b y^2."""
    dx, W = prm["dx"], prm["W"]
    h0 = row_crossing(phi[0], dx, W)
    h1 = row_crossing(phi[1], dx, W)
    h_at0 = (9.0 * h0 - h1) / 8.0
    return (0.5 - h_at0) / prm["amplitude"]
