"""The paper's two 3D ablation findings (Sec. 5, drop coalescence in 3D) on
the CUDA path, in FP64 through the C ABI:

* without the bulk viscosity (eta_b = 0) a pressure checkerboard survives:
  a checkerboard theta = (pi, pi, pi) decays far less than with eta_b = eta,
  and both follow the closed-form RK3 amplification of the linearised flow
  operator (the symbol the oracle is pinned to);
* without the pressure averaging of Eq. gradp-u-p-ave-3d the 3D run blows up:
  a small closed-box bubble in the bench's lattice units (c_s tied to the
  step) matches the oracle while its error mode is small, grows by orders of
  magnitude within 220 steps where the averaged run stays quiet, and is
  reported as GPE2P_EDIVERGED once it overflows.  The GPU only sees the
  NaN/Inf values of an unstable explicit scheme; nothing faults."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2011_00814_gb300 import build, gpe2p, inputs
from tests.fields import field_errors
from tests.test_oracle_pins import _mode_field, flow_symbol, rk3_amplification

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


def test_checkerboard_without_bulk_viscosity_on_the_gpu():
    theta = [math.pi] * 3
    p_end = {}
    for bulk in (0, 1):
        prm = inputs.base_params(3, 4, 4, 4, dx=0.5, dt=0.05, cs=1.3, rhoL=1.7, rhoG=0.4, etaL=0.05, etaG=0.02,
                                 sigma=0.0, M=0.01, W=3.0, bulk_visc=bulk, p_average=1)
        eps, nsteps = 1e-30, 40
        q0 = np.array([1j, 0, 0, 0], dtype=complex)
        f = inputs.zero_fields(prm)
        f["phi"][...] = 1.0
        f["p"] = _mode_field(prm, "c", eps * q0[0], theta)
        with gpe2p.Solver(dict(prm, precision=64)) as s:
            s.init_fields(f)
            s.advance(nsteps)
            out = s.read_fields()
        G = rk3_amplification(prm["dt"] * flow_symbol(prm, theta, 1.0))
        qN = np.linalg.matrix_power(G, nsteps) @ q0
        want = _mode_field(prm, "c", eps * qN[0], theta)
        assert np.max(np.abs(out["p"] - want)) < 1e-11 * eps, bulk
        for c, k in enumerate(("u", "v", "w")):
            want_k = _mode_field(prm, k, eps * qN[1 + c], theta)
            assert np.max(np.abs(out[k] - want_k)) < 1e-11 * eps, (bulk, k)
        p_end[bulk] = float(np.max(np.abs(out["p"]))) / eps
    assert p_end[1] < 0.1 * p_end[0], p_end


def test_3d_bubble_without_pressure_averaging_blows_up_on_the_gpu():
    prm, f = inputs.bubble3d(16, 16, 32, R=5, gap=6)
    prm = dict(prm, check_stability=0, precision=64)
    # the first steps, while the unstable modes are still small, match the oracle
    q = dict(prm, p_average=0)
    n0 = 60
    st = oracle.init_state(q, f["phi"], f["p"], f["u"], f["v"], f["w"])
    ref = oracle.step(q, st, n0)
    Uc = prm["sigma"] / prm["etaL"]
    with gpe2p.Solver(q) as s:
        s.init_fields(f)
        s.advance(n0)
        got = s.read_fields()
        errs = field_errors(q, got, ref, Uc)
        assert max(errs[k] for k in ("phi", "p", "u", "v", "w")) < 1e-11, errs
        # then it grows until it overflows within the oracle pin's 220 steps,
        # and the step reports it; the state stays readable
        grown, step = 0.0, n0
        with pytest.raises(gpe2p.GPE2PError) as e:
            while step < 220:
                s.advance(10)
                step += 10
                pf = s.read_fields()["p"]
                grown = max(grown, float(np.max(np.abs(pf[np.isfinite(pf)]))) if np.any(np.isfinite(pf)) else 0.0)
        assert e.value.code == gpe2p.EDIVERGED
        assert s.diagnostics()["nan_flag"] == 1
    with gpe2p.Solver(dict(prm, p_average=1)) as s:
        s.init_fields(f)
        s.advance(220)
        p_avg = float(np.max(np.abs(s.read_fields()["p"])))
    assert p_avg < 1e-3, p_avg
    # before it overflowed, the unaveraged pressure had grown far past the averaged one
    assert grown > 1e3 * p_avg, (grown, p_avg)
