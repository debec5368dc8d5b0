"""The precision policy of the phi accumulation on FP32 problems.

With the conservative advection form the Cahn-Hilliard update conserves the
phi integral exactly in exact arithmetic (the isotropic Laplacian and the
isotropic divergence of a periodic field sum to zero), so any drift of the
integral is rounding.  In FP32 the rounding of phi + dt L, about 3e-8 per
cell and step, makes the relative drift of the integral grow far past 1e-10
within a few hundred steps; the compensated accumulation (phi as an FP32
high/low pair, the final RK stage in FP64) leaves only the rounding of the
rate itself, orders of magnitude smaller.  The automatic policy switches to
it at the first diagnostics past the threshold."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2011_00814_gb300 import build, gpe2p, inputs

pytestmark = pytest.mark.gpu

STEPS = 400


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


def drop():
    prm, f = inputs.static_drop(n=64, R=16.0)
    prm = dict(prm, precision=32, ch_advection=1, diag_every=20)
    return prm, f


def run(mode, steps=STEPS):
    prm, f = drop()
    with gpe2p.Solver(prm) as s:
        s.set_phi_accumulation(mode, 1e-10)
        s.init_fields(f)
        s.advance(steps)
        st = s.phi_accumulation()
        st["phi"] = s.read_fields()["phi"]
        return st


def test_fp32_accumulation_drifts_and_compensated_does_not():
    off = run(gpe2p.PHI_ACC_FP32)
    on = run(gpe2p.PHI_ACC_COMPENSATED)
    assert not off["active"] and on["active"]
    assert off["drift"] > 1e-9, off["drift"]
    assert on["drift"] < 1e-10 and on["drift"] < off["drift"] / 100, (on["drift"], off["drift"])


def test_auto_switches_past_the_threshold():
    off = run(gpe2p.PHI_ACC_FP32)
    auto = run(gpe2p.PHI_ACC_AUTO)
    assert auto["active"] and 0 < auto["switched_at"] < STEPS
    # after the switch the drift stops growing
    assert auto["drift"] < 0.25 * off["drift"], (auto, off["drift"])


def test_compensated_phi_against_the_oracle():
    """The FP32 run with the compensated accumulation stays within the FP32
    field tolerance of the FP64 oracle, and both keep the phi integral to
    within 1e-10 of its initial value (relative to the integral of |phi_0|;
    each from its own initial state, since rounding phi_0 to FP32 moves the
    integral by more than that)."""
    prm, f = drop()
    steps = 100
    with gpe2p.Solver(prm) as s:
        s.set_phi_accumulation(gpe2p.PHI_ACC_COMPENSATED)
        s.init_fields(f)
        d = s.advance(steps)
        phi = s.read_fields()["phi"]
        drift = s.phi_accumulation()["drift"]
    st = oracle.init_state(prm, f["phi"], f["p"], f["u"], f["v"])
    out = oracle.step(prm, st, steps)
    ref = out["phi"]
    assert np.max(np.abs(phi - ref)) / np.max(np.abs(ref)) < 1e-4
    a0 = np.abs(f["phi"]).sum()
    assert drift < 1e-10
    assert abs(oracle.diag(prm, out)[0] - oracle.diag(prm, st)[0]) / a0 < 1e-10
