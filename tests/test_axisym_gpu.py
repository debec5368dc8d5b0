"""Parity of the axisymmetric form (x = r with the axis at x = 0, y = z) of the CUDA
path with the CPU FP64 oracle, through the C ABI.

Tolerances as for the planar parity tests: FP64 rates 1e-12 and states after many
steps 1e-11 (max relative field error, floors of tests/fields.py); FP32 rates 2e-5,
states 2e-5 after a few steps of random fields and 1e-4 after the drop runs.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2011_00814_gb300 import build, gpe2p, inputs
from tests.fields import field_errors, max_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


CASES = {
    # ragged tiles along both axes; outer wall no-slip, axial walls no-slip
    "noslip": dict(n=(37, 23), bc=("noslip", "noslip", "periodic")),
    "freeslip-periodic-z": dict(n=(40, 19), bc=("freeslip", "periodic", "periodic")),
    "nobulk-noavg": dict(n=(33, 45), bc=("noslip", "freeslip", "periodic"), bulk_visc=0, p_average=0),
    "rk4": dict(n=(70, 9), bc=("freeslip", "noslip", "periodic"), ch_scheme=4),
}


def case_params(name):
    c = dict(CASES[name])
    nx, ny = c.pop("n")
    return inputs.base_params(2, nx, ny, dx=0.5, dt=0.02, cs=1.2, rhoL=1.0, rhoG=0.2, etaL=0.05, etaG=0.01,
                              rho_ref=0.6, sigma=0.03, M=0.02, W=2.0, g=(0.0, -0.02, 0.0), axisym=1, **c)


def _uh(prm, u, axis):
    """cell average of a face component (face n on a wall is zero)"""
    ax = 1 - axis
    up = np.roll(u, -1, ax)
    if prm["bc"][axis] != "periodic":
        sl = [slice(None)] * 2
        sl[ax] = -1
        up[tuple(sl)] = 0.0
    return 0.25 * ((u + up) + (u + up))


def gpu_run(prm, f, nsteps, precision=64):
    with gpe2p.Solver(dict(prm, precision=precision)) as s:
        s.init_fields(f)
        if nsteps:
            s.advance(nsteps)
        return s.read_fields()


def oracle_run(prm, f, nsteps):
    st = oracle.init_state(prm, f["phi"], f["p"], f["u"], f["v"])
    return oracle.step(prm, st, nsteps) if nsteps else st


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [64, 32])
def test_axisym_rates_match_oracle(name, precision):
    prm = case_params(name)
    f = inputs.random_fields(prm, seed=23)
    st = oracle.init_state(prm, f["phi"], f["p"], f["u"], f["v"])
    ref = oracle.flow_rhs(prm, st)
    ref_phi = oracle.ch_rhs(prm, st["phi"], st["mu"], [_uh(prm, st[k], a) for a, k in enumerate("uv")])
    with gpe2p.Solver(dict(prm, precision=precision)) as s:
        s.init_fields(f)
        got = s.eval_rates()
        mu = s.read_fields()["mu"]
    tol = 1e-12 if precision == 64 else 2e-5
    for k, r in zip(("Lp", "Lu", "Lv"), ref):
        assert max_rel_err(got[k], r, 1e-30) < tol, (k, max_rel_err(got[k], r, 1e-30))
    assert max_rel_err(got["Lphi"], ref_phi, 1e-30) < tol
    assert max_rel_err(mu, st["mu"], 1e-30) < tol
    # the axisymmetric terms are not negligible in these fields: the planar
    # rates differ from them by far more than the tolerance
    flat = oracle.flow_rhs(dict(prm, axisym=0), st)
    assert max_rel_err(flat[0], ref[0], 1e-30) > 1e3 * tol


@pytest.mark.parametrize("name", list(CASES))
def test_axisym_steps_match_oracle_fp64(name):
    prm = case_params(name)
    f = inputs.random_fields(prm, seed=7)
    got, ref = gpu_run(prm, f, 12), oracle_run(prm, f, 12)
    errs = field_errors(prm, got, ref, Uc=0.05)
    assert max(errs.values()) < 1e-11, errs


@pytest.mark.parametrize("name", ["noslip", "rk4"])
def test_axisym_steps_match_oracle_fp32(name):
    prm = case_params(name)
    f = inputs.random_fields(prm, seed=7)
    got, ref = gpu_run(prm, f, 12, 32), oracle_run(prm, f, 12)
    errs = field_errors(prm, got, ref, Uc=0.05)
    assert max(errs.values()) < 2e-5, errs


def test_falling_drop_parity():
    """The falling drop at 8 cells per radius (64 x 192), 400 steps."""
    prm, f = inputs.falling_drop(n_l=8, n_t=640)
    n = 400
    ref = oracle_run(prm, f, n)
    Uc = prm["sigma"] / prm["etaL"]
    e64 = field_errors(prm, gpu_run(prm, f, n, 64), ref, Uc)
    assert max(e64.values()) < 1e-11, e64
    e32 = field_errors(prm, gpu_run(prm, f, n, 32), ref, Uc)
    assert max(e32[k] for k in ("phi", "p", "u", "v")) < 1e-4, e32
    # the drop has started to fall: the axial velocity is well above round-off
    assert np.max(np.abs(ref["v"])) > 1e-3


@pytest.mark.parametrize("oh,n_t", [(0.119, 160), (0.3, 800)])
def test_coalescence_parity(oh, n_t):
    """Drop coalescence at 16 cells per radius (48 x 48), 300 steps."""
    prm, f = inputs.drop_coalescence(oh, n_l=16, n_t=n_t)
    n = 300
    ref = oracle_run(prm, f, n)
    e64 = field_errors(prm, gpu_run(prm, f, n, 64), ref, 1.0)
    assert max(e64.values()) < 1e-11, e64
    e32 = field_errors(prm, gpu_run(prm, f, n, 32), ref, 1.0)
    assert max(e32[k] for k in ("phi", "p", "u", "v")) < 1e-4, e32


def test_falling_drop_full_size_fp64():
    """The falling drop at the paper's 50 cells per radius (400 x 1200), 20 steps,
    every cell against the oracle."""
    prm, f = inputs.falling_drop()
    n = 20
    ref = oracle_run(prm, f, n)
    got = gpu_run(prm, f, n, 64)
    errs = field_errors(prm, got, ref, prm["sigma"] / prm["etaL"])
    assert max(errs.values()) < 1e-11, errs


@pytest.mark.parametrize("precision", [32, 64])
def test_axisym_batch_matches_single_instance_bitwise(precision):
    """Axisymmetric and planar instances side by side in one batch follow the
    single-instance path bit for bit."""
    prms, fields = [], []
    for k, name in enumerate(n for n in CASES if n != "rk4"):  # batches take TVD-RK2 only
        prm = dict(case_params(name), precision=precision)
        prms.append(prm)
        fields.append(inputs.random_fields(prm, seed=60 + k))
    planar = dict(case_params("noslip"), axisym=0, precision=precision)
    prms.append(planar)
    fields.append(inputs.random_fields(planar, seed=99))
    prm, f = inputs.drop_coalescence(0.119, n_l=16, n_t=160, precision=precision)
    prms.append(prm)
    fields.append(f)
    n = 9
    with gpe2p.Batch(prms) as b:
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
