"""Interface positions from a phase field on the cell centres, shared by the
tests: the capillary wave's height at its symmetry plane y = 0, and the
bubble and spike tips of the Rayleigh-Taylor interface."""
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


def column_crossing(col, dy, from_top):
    """y of the phi = 0 crossing of one column (cell centres at (j + 1/2) dy),
    linearly interpolated between the two cells around the sign change: the
    topmost crossing (from_top) or the lowest one, or None if phi keeps its
    sign."""
    s = np.nonzero(np.sign(col[:-1]) != np.sign(col[1:]))[0]
    if s.size == 0:
        return None
    j = int(s[-1] if from_top else s[0])
    a, b = float(col[j]), float(col[j + 1])
    return (j + 0.5) * dy + a / (a - b) * dy


def rt_tips(phi, dx):
    """Bubble and spike tip heights of the Rayleigh-Taylor interface
    y = 2 + 0.1 cos(2 pi x) on a periodic unit width (phi > 0 heavy, on top).
    The bubble of light fluid rises on the column x = 0, the spike of heavy
    fluid falls on x = 1/2; both columns lie on cell faces, so phi there is the
    mean of the two cell columns beside it.  The bubble tip is the topmost
    crossing on x = 0, the spike tip the lowest one on x = 1/2."""
    ny, nx = phi.shape
    c0 = 0.5 * (phi[:, nx - 1] + phi[:, 0])
    c5 = 0.5 * (phi[:, nx // 2 - 1] + phi[:, nx // 2])
    return column_crossing(c0, dx, True), column_crossing(c5, dx, False)
