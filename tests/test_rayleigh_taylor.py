"""The Rayleigh-Taylor tip positions (tests/interface_position.py) on fields
whose tips are known: the initial interface y = 2 + 0.1 cos(2 pi x) of the
workload, a mirrored copy of it, and a column that crosses zero several
times."""
from __future__ import annotations

import math

import numpy as np

from interface_position import column_crossing, rt_tips
from paper_2011_00814_gb300 import inputs


def test_tips_of_the_initial_interface():
    # phi = tanh(2 (y - h(x)) / W): the two face columns x = 0 and 1/2 average
    # the cell columns at x = +-dx/2 around them, whose heights are
    # 2 +- 0.1 cos(pi dx); the linear interpolation of the odd tanh profile
    # across its zero is exact to a small fraction of a cell
    prm, f = inputs.rayleigh_taylor(variant="paper")
    dx = prm["dx"]
    bubble, spike = rt_tips(f["phi"], dx)
    c = 0.1 * math.cos(math.pi * dx)
    assert abs(bubble - (2.0 + c)) < 0.02 * dx
    assert abs(spike - (2.0 - c)) < 0.02 * dx


def test_tips_follow_a_shifted_and_mirrored_field():
    prm, f = inputs.rayleigh_taylor(nx=64, ny=256, variant="paper")
    dx = prm["dx"]
    b0, s0 = rt_tips(f["phi"], dx)
    # shifting the field up by three cells moves both tips by three cells
    up = np.concatenate([np.ones((3, 64)) * -1.0, f["phi"][:-3]], axis=0)
    b1, s1 = rt_tips(up, dx)
    assert abs(b1 - b0 - 3 * dx) < 1e-12 and abs(s1 - s0 - 3 * dx) < 1e-12
    # the half-period shift x -> x + 1/2 exchanges the two columns: the bubble
    # column now carries the lower crossing and the spike column the upper one
    sh = np.roll(f["phi"], 32, axis=1)
    b2, s2 = rt_tips(sh, dx)
    assert abs(b2 - s0) < 1e-12 and abs(s2 - b0) < 1e-12


def test_topmost_and_lowest_crossings_of_a_rolled_up_column():
    # light fluid (phi < 0) in the bands [1, 2) and [3, 5) of a unit-spaced
    # column: crossings at 1, 2, 3 and 5; the bubble tip is the topmost, the
    # spike tip the lowest
    y = np.arange(8) + 0.5
    col = np.where(((y >= 1) & (y < 2)) | ((y >= 3) & (y < 5)), -1.0, 1.0)
    assert column_crossing(col, 1.0, True) == 5.0
    assert column_crossing(col, 1.0, False) == 1.0
    assert column_crossing(np.ones(8), 1.0, True) is None
