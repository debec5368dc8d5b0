"""The seeded workloads carry the dimensionless numbers of the paper's cases
(Sec. "Falling drop", Sec. "Drop coalescence (axisymmetric)", Sec. "Capillary
wave in 2D") and the discretisation convention of Sec. 4 (dx = L_c / N_L,
dt = T_c / N_t, c_s = (dx / dt) / sqrt 3 with U_c = sigma / eta_L)."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2011_00814_gb300 import inputs


def _speeds(prm, Lc=1.0):
    Uc = prm["sigma"] / prm["etaL"]
    Tc = Lc / Uc
    return Uc, Tc


def test_falling_drop_numbers():
    prm, f = inputs.falling_drop()
    R, D = 1.0, 2.0
    drho = prm["rhoL"] - prm["rhoG"]
    assert abs(prm["rhoL"] / prm["rhoG"] - 1.15) < 1e-12
    assert prm["etaL"] == prm["etaG"]
    assert abs(prm["g"][1] * drho * D * D / prm["sigma"] - 144.0) < 1e-9
    assert abs(prm["etaL"] / math.sqrt(prm["rhoL"] * D * prm["sigma"]) - 0.0466) < 1e-12
    assert prm["rho_ref"] == prm["rhoG"] and prm["g"][0] == 0.0
    Uc, Tc = _speeds(prm, R)
    assert abs(prm["dx"] - R / 50) < 1e-15 and abs(prm["dt"] - Tc / 4000) < 1e-15
    assert abs(prm["cs"] - (prm["dx"] / prm["dt"]) / math.sqrt(3.0)) < 1e-12
    assert (prm["nx"], prm["ny"]) == (400, 1200) and prm["axisym"] == 1
    assert abs(prm["W"] - 0.06 * R) < 1e-15 and abs(prm["M"] - 1.0 / 1000.0) < 1e-15
    # the drop: phi > 0 inside r_dc < R around (z, r) = (2, 0), tanh profile of width Cn
    r, z = inputs.cell_centres(prm)
    inside = np.hypot(z - 2.0, r) < R - 3 * prm["W"]
    outside = np.hypot(z - 2.0, r) > R + 3 * prm["W"]
    assert np.all(f["phi"][inside] > 0.99) and np.all(f["phi"][outside] < -0.99)


@pytest.mark.parametrize("oh,nt", [(0.037, 400), (0.119, 400), (0.3, 2000)])
def test_drop_coalescence_numbers(oh, nt):
    prm, f = inputs.drop_coalescence(oh)
    assert abs(prm["rhoL"] / prm["rhoG"] - 50.0) < 1e-12
    assert abs(prm["etaL"] / prm["etaG"] - 58.8) < 1e-12
    assert abs(prm["etaL"] / math.sqrt(prm["rhoL"] * prm["sigma"] * 1.0) - oh) < 1e-12
    Uc, Tc = _speeds(prm)
    assert abs(prm["dt"] - Tc / nt) < 1e-15 and (prm["nx"], prm["ny"]) == (120, 120)
    assert prm["bc"][:2] == ("freeslip", "freeslip") and prm["axisym"] == 1
    # the drop touches the mirror plane z = 0 on the axis
    r, z = inputs.cell_centres(prm)
    assert f["phi"][0, 0] > 0.0


@pytest.mark.parametrize("n,nt,cn,pe", [(64, 384, 0.0625, 2e4), (128, 1920, 0.03125, 4e4)])
def test_capillary_wave_numbers(n, nt, cn, pe):
    prm, f = inputs.capillary_wave(n, nt, cn, pe)
    Uc, Tc = _speeds(prm)
    assert abs(Uc - 1.0) < 1e-15
    assert abs(prm["rhoL"] * Uc * 1.0 / prm["etaL"] - 1000.0) < 1e-9  # Re
    assert abs(prm["rhoL"] / prm["rhoG"] - 20.0) < 1e-12 and abs(prm["etaL"] / prm["etaG"] - 20.0) < 1e-12
    assert abs(prm["dx"] - 1.0 / n) < 1e-15 and abs(prm["dt"] - Tc / nt) < 1e-15
    assert abs(prm["W"] - cn) < 1e-15 and abs(prm["M"] - 1.0 / pe) < 1e-15
