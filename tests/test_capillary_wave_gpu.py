"""The capillary wave on the GPU: FP64 parity with the oracle over the first
768 steps, and the paper's validation against the closed form (Eq.
cap-wave-analytical) over 0 <= t <= 30 on its coarse and fine meshes, where
the deviation must stay small and shrink with refinement."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import capillary as C
from paper_2011_00814_gb300 import build, gpe2p, inputs

from interface_position import h_tilde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


def test_fp64_parity_with_the_oracle():
    prm, f = inputs.capillary_wave()
    n = 768
    with gpe2p.Solver(prm) as s:
        s.init_fields(f)
        s.advance(n)
        got = s.read_fields()
    ref = oracle.step(prm, oracle.init_state(prm, f["phi"], f["p"], f["u"], f["v"]), n)
    for key, floor in (("phi", 1.0), ("u", 1.0), ("v", 1.0), ("p", 1.0), ("mu", 3.0 / prm["W"])):
        err = np.max(np.abs(got[key] - ref[key])) / max(np.max(np.abs(ref[key])), 1e-3 * floor)
        assert err < 1e-11, (key, err)


def deviation(n, nt, cn, pe, precision, t_end=30.0):
    prm, f = inputs.capillary_wave(n, nt, cn, pe, precision)
    steps = int(round(nt / 4))                 # a quarter of T_c
    ts, hs = [], []
    with gpe2p.Solver(prm) as s:
        s.init_fields(f)
        for m in range(1, int(round(4 * t_end)) + 1):
            s.advance(steps)
            ts.append(m * steps * prm["dt"])
            hs.append(h_tilde(s.read_fields()["phi"], prm))
    ex = C.h_tilde(np.array(ts), prm["sigma"], prm["rhoL"], prm["rhoG"], prm["etaL"] / prm["rhoL"], 2.0 * math.pi)
    return float(np.max(np.abs(np.array(hs) - ex)))


@pytest.mark.parametrize("precision", [64, 32])
def test_closed_form_and_refinement(precision):
    coarse = deviation(64, 384, 0.0625, 2.0e4, precision)
    fine = deviation(128, 1920, 0.03125, 4.0e4, precision)
    assert coarse < 0.15, coarse
    assert fine < 0.7 * coarse, (coarse, fine)
