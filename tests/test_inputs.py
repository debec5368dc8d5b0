"""The seeded workloads carry the parameter sets the paper prints for its
cases (`tests/golden/paper_parameters.json`, each entry citing its passage):
the dimensionless numbers and the discretisation convention of Sec. 4 (dx =
L_c / N_L, dt = T_c / N_t, c_s = (dx / dt) / sqrt 3, U_c = sigma / eta_L)."""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

from paper_2011_00814_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


def _check_discretisation(prm, g, n_t, Lc=1.0):
    Uc = prm["sigma"] / prm["etaL"]
    Tc = Lc / Uc
    assert abs(prm["dx"] - Lc / g["N_L"]) < 1e-15
    assert abs(prm["dt"] - Tc / n_t) < 1e-15
    assert abs((prm["dx"] / prm["dt"]) / Uc - n_t / g["N_L"]) < 1e-9  # c
    assert abs(prm["cs"] - (prm["dx"] / prm["dt"]) / math.sqrt(3.0)) < 1e-12
    assert abs(prm["W"] - g["Cn"] * Lc) < 1e-15
    assert abs(prm["M"] - Uc * Lc / g["Pe"]) < 1e-15


def test_falling_drop_numbers():
    g = GOLDEN["falling_drop"]
    prm, f = inputs.falling_drop()
    R, D = 1.0, 2.0
    drho = prm["rhoL"] - prm["rhoG"]
    assert abs(prm["rhoL"] / prm["rhoG"] - g["r_rho"]) < 1e-12
    assert abs(prm["etaL"] / prm["etaG"] - g["r_eta"]) < 1e-12
    assert abs(prm["g"][1] * drho * D * D / prm["sigma"] - g["Eo"]) < 1e-9
    assert abs(prm["etaL"] / math.sqrt(prm["rhoL"] * D * prm["sigma"]) - g["Oh"]) < 1e-12
    assert prm["rho_ref"] == prm["rhoG"] and prm["g"][0] == 0.0
    assert g["N_t"] / g["N_L"] == g["c"]
    _check_discretisation(prm, g, g["N_t"], R)
    assert (prm["nx"], prm["ny"]) == (g["L_r"] * g["N_L"], g["L_z"] * g["N_L"]) and prm["axisym"] == 1
    # the drop: phi > 0 inside r_dc < R around (z, r) = (z_c, 0), tanh profile of width Cn
    r, z = inputs.cell_centres(prm)
    inside = np.hypot(z - g["z_c"], r) < R - 3 * prm["W"]
    outside = np.hypot(z - g["z_c"], r) > R + 3 * prm["W"]
    assert np.all(f["phi"][inside] > 0.99) and np.all(f["phi"][outside] < -0.99)


@pytest.mark.parametrize("oh", GOLDEN["drop_coalescence"]["Oh"])
def test_drop_coalescence_numbers(oh):
    g = GOLDEN["drop_coalescence"]
    prm, f = inputs.drop_coalescence(oh)
    assert abs(prm["rhoL"] / prm["rhoG"] - g["r_rho"]) < 1e-12
    assert abs(prm["etaL"] / prm["etaG"] - g["r_eta"]) < 1e-12
    assert abs(prm["etaL"] / math.sqrt(prm["rhoL"] * prm["sigma"] * 1.0) - oh) < 1e-12
    n_t = g["N_t"][str(oh)]
    assert n_t / g["N_L"] == g["c"][str(oh)]
    _check_discretisation(prm, g, n_t)
    assert (prm["nx"], prm["ny"]) == (g["L_r"] * g["N_L"], g["L_z"] * g["N_L"])
    assert prm["bc"][:2] == ("freeslip", "freeslip") and prm["axisym"] == 1
    # the drop touches the mirror plane z = 0 on the axis
    assert f["phi"][0, 0] > 0.0


@pytest.mark.parametrize("case", ["capillary_wave_coarse", "capillary_wave_fine"])
def test_capillary_wave_numbers(case):
    g = GOLDEN[case]
    prm, f = inputs.capillary_wave(g["N_L"], g["N_t"], g["Cn"], g["Pe"])
    assert abs(prm["sigma"] / prm["etaL"] - 1.0) < 1e-15
    assert abs(prm["rhoL"] * 1.0 * 1.0 / prm["etaL"] - g["Re"]) < 1e-9
    assert abs(prm["rhoL"] / prm["rhoG"] - g["r_rho"]) < 1e-12
    assert abs(prm["etaL"] / prm["etaG"] - g["r_eta"]) < 1e-12
    assert abs(prm["amplitude"] - g["A_p"]) < 1e-15
    assert g["N_t"] / g["N_L"] == g["c"]
    _check_discretisation(prm, g, g["N_t"])
