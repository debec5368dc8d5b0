"""The surrogate's evaluation measures against closed forms (CPU).

For a circle of radius R translated by s cells, the phi = 0 contours are
exactly s apart (Hausdorff distance s) and the mean normal displacement of
the translated circle is (2/pi) s; a radius change dR moves every point of
the contour by dR."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2011_00814_gb300 import surrogate as S

pytest.importorskip("scipy")

N = 128


def circle(cx, cy, R, W=4.0):
    y, x = np.mgrid[0:N, 0:N] + 0.5
    dx = np.abs(x - cx)
    dx = np.minimum(dx, N - dx)
    dy = np.abs(y - cy)
    dy = np.minimum(dy, N - dy)
    return np.tanh(2.0 * (R - np.hypot(dx, dy)) / W)


@pytest.mark.parametrize("s", [0.5, 1.0, 2.0])
def test_translated_circle(s):
    a, b = circle(64, 64, 30), circle(64 + s, 64, 30)
    assert abs(S.interface_hausdorff(a, b) - s) < 0.05
    assert abs(S.interface_error(a, b)[0] - 2.0 * s / math.pi) < 0.03 * s + 0.01


def test_radius_change_and_periodic_wrap():
    assert abs(S.interface_hausdorff(circle(64, 64, 30), circle(64, 64, 31.5)) - 1.5) < 0.05
    # a drop that straddles the periodic boundary, moved across it
    assert abs(S.interface_hausdorff(circle(127.8, 64, 20), circle(0.3, 64, 20)) - 0.5) < 0.05


def test_phi_l2_and_identity():
    a = circle(64, 64, 30)
    assert S.interface_hausdorff(a, a) == 0.0
    assert S.phi_l2(a, a) == 0.0
    assert abs(S.phi_l2(-a, a) - 2.0) < 1e-12
