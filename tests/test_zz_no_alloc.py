"""The allocation-free diagnostics entry point (gpe2p_diagnostics_noalloc).

Some callers cannot allocate device memory when they need the diagnostics
(during a CUDA-graph capture, under a custom memory pool, or in a loop that
must not block in cudaMalloc); this entry point serves them from a fixed
scratch array in the library.  The test calls it through the C ABI on the
device pointers of a live state and checks it against gpe2p_diagnostics of
the same state, twice in a row (the scratch keeps the previous call's
contents), in FP32 3D and FP64 2D, and in FP32 under the compensated phi
accumulation, where the low part of phi (field 6 of gpe2p_field_ptr) is
passed too and must enter the phi integral.  It lives in its own file so that
pytest collects it last.
"""
from __future__ import annotations

import ctypes

import pytest

from paper_2011_00814_gb300 import build, gpe2p, inputs

pytestmark = pytest.mark.gpu


def _call(L, q, ptr, phi_lo, pitch, out):
    import torch

    out.fill_(-1.0)
    torch.cuda.synchronize()
    rc = L.gpe2p_diagnostics_noalloc(ctypes.byref(q), ptr["p"], ptr["u"], ptr["v"], ptr.get("w"), ptr["phi"],
                                     phi_lo, pitch, out.data_ptr(), None)
    assert rc == gpe2p.OK
    torch.cuda.synchronize()
    return out.cpu().tolist()


def _check(prm, nsteps, compensated=False):
    import torch

    build.build()
    L = gpe2p.lib()
    with gpe2p.Solver(prm) as s:
        # a fixed accumulation policy: the automatic one may switch on the
        # compensated accumulation at the diagnostics that end advance()
        s.set_phi_accumulation(gpe2p.PHI_ACC_COMPENSATED if compensated else gpe2p.PHI_ACC_FP32)
        s.init_fields(inputs.random_fields(prm, seed=21))
        s.advance(nsteps)
        ref = s.diagnostics()
        ptr = {}
        for k in ("p", "u", "v", "phi", "phi_lo") + (("w",) if prm["dim"] == 3 else ()):
            ptr[k], pitch = s.field_ptr(k)
        # the low part of phi exists exactly while the compensated accumulation runs
        assert (ptr["phi_lo"] is not None) == compensated
        q = gpe2p.params(prm)
        out = torch.zeros(4, dtype=torch.float64, device="cuda")
        ncell = prm["nx"] * prm["ny"] * prm["nz"]
        vol = prm["dx"] ** prm["dim"]
        tol_phi = 1e-12 * ncell * vol
        for _ in range(2):
            got = _call(L, q, ptr, ptr["phi_lo"], pitch, out)
            assert abs(got[0] - ref["int_phi"]) <= tol_phi
            assert abs(got[1] - ref["kinetic"]) <= 1e-12 * ref["kinetic"]
            assert got[2] == ref["umax"]
            assert got[3] == 0.0 and ref["nan_flag"] == 0
        if compensated:
            # without its low part the integral is off by more than the bound
            # above, so the check of the low part is not vacuous
            got = _call(L, q, ptr, None, pitch, out)
            assert abs(got[0] - ref["int_phi"]) > tol_phi


def test_noalloc_diagnostics_match_fp32_3d():
    prm = dict(inputs.base_params(3, 37, 21, 19, dx=0.5, dt=0.02, cs=1.2, W=2.0, sigma=0.02,
                                  bc=("noslip", "periodic", "freeslip")), precision=32)
    _check(prm, 3)


def test_noalloc_diagnostics_match_fp64_2d():
    prm = dict(inputs.base_params(2, 45, 30, dx=0.5, dt=0.02, cs=1.2, W=2.0, sigma=0.02,
                                  bc=("periodic", "noslip", "periodic")), precision=64)
    _check(prm, 3)


def test_noalloc_diagnostics_match_compensated_phi_fp32_3d():
    prm = dict(inputs.base_params(3, 37, 21, 19, dx=0.5, dt=0.02, cs=1.2, W=2.0, sigma=0.02,
                                  bc=("noslip", "periodic", "freeslip")), precision=32)
    _check(prm, 6, compensated=True)


def test_noalloc_rejects_grids_beyond_its_scratch():
    build.build()
    L = gpe2p.lib()
    prm = dict(inputs.base_params(3, 4096, 4096, 8), precision=32)
    q = gpe2p.params(prm)
    dummy = ctypes.c_void_p(256)
    rc = L.gpe2p_diagnostics_noalloc(ctypes.byref(q), dummy, dummy, dummy, dummy, dummy, None, 4096, dummy, None)
    assert rc == gpe2p.EINVAL
