"""The oracle against the closed-form capillary wave (Sec. "Capillary wave in
2D", Eq. cap-wave-analytical), CPU.

The closed form itself is pinned at t = 0 (h~ = 1) and in the inviscid limit
(h~ -> cos(omega_0 t)).  The oracle, run on the paper's coarse mesh (N_L = 64,
N_t = 384, Cn = 0.0625, Pe = 2 10^4), follows it over the first half period
to within 0.1 of the initial amplitude: the paper reports agreement in the
early stage with deviations that grow slowly and shrink with refinement (its
figure data are not available; the refinement is checked on the GPU)."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import capillary as C
from paper_2011_00814_gb300 import inputs

from interface_position import h_tilde

pytest.importorskip("scipy")


def test_closed_form_at_zero_and_inviscid_limit():
    k = 2.0 * math.pi
    assert abs(C.h_tilde(np.array([0.0]), 1e-3, 1.0, 0.05, 1e-3, k)[0] - 1.0) < 1e-12
    w0 = C.omega0_of(1e-3, 1.0, 0.05, k)
    t = np.linspace(0.0, 20.0, 9)
    assert np.max(np.abs(C.h_tilde(t, 1e-3, 1.0, 0.05, 1e-12, k) - np.cos(w0 * t))) < 1e-4


def test_oracle_follows_the_closed_form_early():
    prm, f = inputs.capillary_wave()
    st = oracle.init_state(prm, f["phi"], f["p"], f["u"], f["v"])
    assert abs(h_tilde(st["phi"], prm) - 1.0) < 1e-4
    ts, hs = [], []
    for m in range(1, 25):                     # t = 0.25 .. 6
        st = oracle.step(prm, st, 96)
        ts.append(m * 96 * prm["dt"])
        hs.append(h_tilde(st["phi"], prm))
    ex = C.h_tilde(np.array(ts), prm["sigma"], prm["rhoL"], prm["rhoG"], prm["etaL"] / prm["rhoL"], 2.0 * math.pi)
    assert np.max(np.abs(np.array(hs) - ex)) < 0.1
