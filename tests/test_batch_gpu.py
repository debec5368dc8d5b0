"""The batched 2D engine: every instance of a batch follows the
single-instance path bit for bit (same per-tile device code), in both the
persistent and the per-sweep form, and the instances match the oracle; a
grid barrier that is made to time out reports GPE2P_ETIMEOUT without
hanging, and the handle recovers after the switch is cleared."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2011_00814_gb300 import build, gpe2p, inputs
from tests.fields import field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


def small_batch(precision):
    specs = [((37, 23), ("periodic", "periodic"), 0), ((64, 64), ("noslip", "freeslip"), 0),
             ((40, 19), ("freeslip", "noslip"), 1), ((96, 50), ("periodic", "noslip"), 0),
             ((33, 17), ("noslip", "periodic"), 1)]
    prms, fields = [], []
    for k, ((nx, ny), bc, cons) in enumerate(specs):
        prm = inputs.base_params(2, nx, ny, dx=0.5, dt=0.02, cs=1.2, rhoL=1.0, rhoG=0.2 + 0.1 * k, etaL=0.05,
                                 etaG=0.01, rho_ref=0.6, sigma=0.03, M=0.02, W=2.0, g=(0.01, -0.02 * k, 0.0),
                                 bc=bc + ("periodic",), ch_advection=cons)
        prm["precision"] = precision
        prms.append(prm)
        fields.append(inputs.random_fields(prm, seed=40 + k))
    return prms, fields


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_matches_single_instance_bitwise(precision, persistent):
    prms, fields = small_batch(precision)
    n = 9
    with gpe2p.Batch(prms) as b:
        b.fault(gpe2p.FAULT_FORCE_PERSISTENT, persistent)
        for k, f in enumerate(fields):
            b.init_instance(k, f)
        b.advance(n)
        got = [b.read_instance(k) for k in range(len(prms))]
    for k, (prm, f) in enumerate(zip(prms, fields)):
        with gpe2p.Solver(prm) as s:
            s.init_fields(f)
            s.advance(n)
            ref = s.read_fields()
        for key in ("phi", "p", "u", "v", "mu"):
            assert np.array_equal(got[k][key], ref[key]), (k, key)


def test_batch_instances_match_oracle_fp64():
    prms, fields = small_batch(64)
    n = 6
    with gpe2p.Batch(prms) as b:
        for k, f in enumerate(fields):
            b.init_instance(k, f)
        b.advance(n)
        for k in (0, 2, 4):
            got = b.read_instance(k)
            st = oracle.init_state(prms[k], fields[k]["phi"], fields[k]["p"], fields[k]["u"], fields[k]["v"])
            ref = oracle.step(prms[k], st, n)
            errs = field_errors(prms[k], got, ref, Uc=0.05)
            assert max(errs.values()) < 1e-11, (k, errs)
            d = b.diagnostics(k)
            assert abs(d["int_phi"] - oracle.diag(prms[k], ref)[0]) < 1e-9


def test_autotuner_reports_a_configuration():
    prms, fields = small_batch(32)
    with gpe2p.Batch(prms) as b:
        c = b.config()
    assert c["tile"] in ((32, 8), (64, 4), (16, 16))
    assert c["tuned_ms_per_step"] > 0.0


def test_barrier_timeout_is_reported_and_recovers():
    prms, fields = small_batch(32)
    with gpe2p.Batch(prms) as b:
        b.fault(gpe2p.FAULT_FORCE_PERSISTENT, 1)
        for k, f in enumerate(fields):
            b.init_instance(k, f)
        b.fault(gpe2p.FAULT_WAIT_LIMIT, 2_000_000)      # about a millisecond of SM clock
        b.fault(gpe2p.FAULT_SKIP_BARRIER, 0)            # block 0 never arrives
        with pytest.raises(gpe2p.GPE2PError) as e:
            b.advance(2)
        assert e.value.code == gpe2p.ETIMEOUT
        b.fault(gpe2p.FAULT_CLEAR)
        for k, f in enumerate(fields):
            b.init_instance(k, f)
        d = b.advance(3)
        assert d["nan_flag"] == 0


def test_uneven_batch_workload_steps_without_divergence():
    prms, fields = inputs.batch_instances(n=12, seed=3)
    with gpe2p.Batch(prms) as b:
        for k, f in enumerate(fields):
            b.init_instance(k, f)
        d = b.advance(20)
        assert d["nan_flag"] == 0
        for k in range(len(prms)):
            dk = b.diagnostics(k)
            s0 = float(np.sum(fields[k]["phi"]))
            assert abs(dk["int_phi"] - s0) < 1e-3 * np.sum(np.abs(fields[k]["phi"]))
