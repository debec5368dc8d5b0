"""Host-side checks of the C ABI: the library builds, loads and exports every
entry point the header declares, the ctypes structs match the C layout, and
the host-only entry points (validation, stability limits) behave."""
from __future__ import annotations

import ctypes
import math
import os
import re
import subprocess

import pytest

from paper_2011_00814_gb300 import build, gpe2p, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpe2p.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gpe2p.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gpe2p_[a-z_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for nm in ("gpe2p_create", "gpe2p_init_fields", "gpe2p_step", "gpe2p_advance", "gpe2p_read_fields",
               "gpe2p_destroy", "gpe2p_last_error", "gpe2p_stability_limits"):
        assert nm in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gpe2p.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for nm in declared_functions():
        assert nm in exported, nm
        assert hasattr(lib, nm)


def _c_layout():
    """sizeof / offsetof of the header structs, from a C compiler."""
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "gpe2p.h"
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("gpe2p_params %zu\n", sizeof(gpe2p_params));
  printf("gpe2p_diag %zu\n", sizeof(gpe2p_diag));
  O(gpe2p_params, dx); O(gpe2p_params, g); O(gpe2p_params, bc); O(gpe2p_params, precision);
  O(gpe2p_params, diag_every); O(gpe2p_params, axisym); O(gpe2p_diag, nan_flag); O(gpe2p_diag, step); O(gpe2p_diag, t);
  return 0;
}
"""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return dict((k, int(v)) for k, v in (line.split() for line in out.splitlines()))


def test_ctypes_structs_match_header_layout():
    lay = _c_layout()
    assert lay["gpe2p_params"] == ctypes.sizeof(gpe2p.Params)
    assert lay["gpe2p_diag"] == ctypes.sizeof(gpe2p.Diag)
    for f in ("dx", "g", "bc", "precision", "diag_every", "axisym"):
        assert lay[f"gpe2p_params.{f}"] == getattr(gpe2p.Params, f).offset, f
    for f in ("nan_flag", "step", "t"):
        assert lay[f"gpe2p_diag.{f}"] == getattr(gpe2p.Diag, f).offset, f


def test_stability_limits_of_the_workloads(lib):
    # the static drop: margins of the reading (acoustic c_s dt/dx = 0.3)
    prm, _ = inputs.static_drop()
    ac, vi, ch = gpe2p.stability_limits(prm)
    assert prm["dt"] < ac and prm["dt"] < vi and prm["dt"] < ch
    # acoustic limit of the 2D staggered operator with averaging: sqrt(3)/2 dx/c_s
    assert abs(ac - math.sqrt(3.0) / 2.0) < 1e-12
    # the 3D bubble is stable only because of the pressure averaging (Sec. 4.5)
    prm, _ = inputs.bubble3d(32, 32, 64, R=8, gap=8)
    ac, vi, ch = gpe2p.stability_limits(prm)
    assert prm["dt"] < min(ac, vi, ch)
    ac0, _, _ = gpe2p.stability_limits(dict(prm, p_average=0))
    assert prm["dt"] > ac0
    # the axisymmetric workloads at the paper's resolutions
    for prm, _ in (inputs.falling_drop(), inputs.drop_coalescence(0.037), inputs.drop_coalescence(0.119),
                   inputs.drop_coalescence(0.3)):
        assert prm["dt"] < min(gpe2p.stability_limits(prm))
    # the Rayleigh-Taylor case at Pe = 1000: the CH limit sets dt
    prm, _ = inputs.rayleigh_taylor()
    ac, vi, ch = gpe2p.stability_limits(prm)
    assert prm["dt"] < ch < 2.5 * prm["dt"]


@pytest.mark.parametrize("bad", [dict(dim=4), dict(nx=0), dict(nx=70000), dict(dx=0.0), dict(dt=-1.0),
                                 dict(rhoG=0.0), dict(etaL=-1.0), dict(W=0.0), dict(precision=16),
                                 dict(ch_scheme=3), dict(iso=15), dict(bc=("wall",) * 3),
                                 dict(bulk_visc=2), dict(sigma=float("nan")), dict(axisym=2),
                                 # the axisymmetric form: 2D, an outer wall, advective CH, axial g
                                 dict(axisym=1, dim=3, nz=8, iso=15, bc=("noslip",) * 3),
                                 dict(axisym=1, bc=("periodic", "noslip", "periodic")),
                                 dict(axisym=1, bc=("noslip",) * 3, ch_advection=1),
                                 dict(axisym=1, bc=("noslip",) * 3, g=(0.1, 0.0, 0.0))])
def test_invalid_parameters_are_rejected_on_the_host(lib, bad):
    prm = dict(inputs.base_params(2, 8, 8), precision=64)
    if bad.get("bc") == ("wall",) * 3:
        q = gpe2p.params(prm)
        q.bc[0] = 7
        out = (ctypes.c_double * 3)()
        assert lib.gpe2p_stability_limits(ctypes.byref(q), out) == gpe2p.EINVAL
        return
    prm.update(bad)
    with pytest.raises(gpe2p.GPE2PError) as e:
        gpe2p.stability_limits(prm)
    assert e.value.code == gpe2p.EINVAL


def test_null_arguments_do_not_crash(lib):
    assert lib.gpe2p_set_phi_accumulation(None, gpe2p.PHI_ACC_AUTO, 1e-10) == gpe2p.EINVAL
    assert lib.gpe2p_phi_accumulation(None, None, None, None, None) == gpe2p.EINVAL
    assert lib.gpe2p_step(None) == gpe2p.EINVAL
    assert lib.gpe2p_advance(None, 1, None) == gpe2p.EINVAL
    assert lib.gpe2p_read_fields(None, None, None, None, None, None, None) == gpe2p.EINVAL
    lib.gpe2p_destroy(None)
    h = ctypes.c_void_p()
    assert lib.gpe2p_create(None, None, ctypes.byref(h)) == gpe2p.EINVAL
    assert b"NULL" in lib.gpe2p_last_error(None)


def test_create_refuses_unstable_dt_before_touching_the_device(lib):
    """With check_stability = 1, gpe2p_create and gpe2p_create_batch compare dt
    with each explicit limit and refuse on the host (no device is needed to
    reach the refusal), naming the limit or the instance."""
    prm = dict(inputs.base_params(2, 16, 16), precision=64, check_stability=1)
    lim = gpe2p.stability_limits(prm)
    names = ("acoustic", "viscous", "Cahn-Hilliard")
    for which in range(3):
        # make limit `which` the binding one and step just past it
        q = dict(prm)
        if which == 0:
            q.update(cs=50.0)
        elif which == 1:
            q.update(etaL=5.0, etaG=0.5)
        else:
            q.update(M=5.0)
        lims = gpe2p.stability_limits(q)
        assert min(range(3), key=lambda t: lims[t]) == which
        q["dt"] = 1.01 * lims[which]
        with pytest.raises(gpe2p.GPE2PError) as e:
            gpe2p.Solver(q)
        assert e.value.code == gpe2p.EUNSTABLE and names[which] in str(e.value)
        with pytest.raises(gpe2p.GPE2PError) as e:
            gpe2p.Batch([prm, q])
        assert e.value.code == gpe2p.EUNSTABLE and "instance 1" in str(e.value)
    assert prm["dt"] < min(lim)


def test_create_batch_validates_every_instance(lib):
    good = dict(inputs.base_params(2, 16, 16), precision=32)
    with pytest.raises(gpe2p.GPE2PError) as e:
        gpe2p.Batch([good, good, dict(good, W=-1.0)])
    assert e.value.code == gpe2p.EINVAL and "instance 2" in str(e.value)
    h = ctypes.c_void_p()
    arr = (gpe2p.Params * 1)(gpe2p.params(good))
    assert lib.gpe2p_create_batch(arr, 0, None, ctypes.byref(h)) == gpe2p.EINVAL
    assert lib.gpe2p_create_batch(None, 1, None, ctypes.byref(h)) == gpe2p.EINVAL


def test_noalloc_diagnostics_validate_on_the_host(lib):
    """gpe2p_diagnostics_noalloc checks its arguments before it looks up its
    scratch or launches anything.  Run only where no GPU is visible, so that
    the one well-formed call below ends at the device lookup (GPE2P_ECUDA)
    and its stand-in pointers are never read."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a visible GPU")
    f = lib.gpe2p_diagnostics_noalloc
    fake = ctypes.c_void_p(4096)
    out = ctypes.cast(ctypes.c_void_p(8192), ctypes.POINTER(ctypes.c_double))

    def call(prm, pitch=None, w=fake, outp=out, p=fake):
        q = gpe2p.params(prm)
        pitch = prm["nx"] if pitch is None else pitch
        return f(ctypes.byref(q), p, fake, fake, w, fake, None, pitch, outp, None)

    good3 = dict(inputs.base_params(3, 8, 6, 4), precision=32)
    good2 = dict(inputs.base_params(2, 8, 6), precision=64)
    assert call(good3, w=None) == gpe2p.EINVAL              # 3D needs w
    assert call(good2, p=None) == gpe2p.EINVAL
    assert call(good2, outp=None) == gpe2p.EINVAL
    assert call(good2, pitch=7) == gpe2p.EINVAL              # row pitch below nx
    assert call(dict(good2, precision=16)) == gpe2p.EINVAL
    assert call(dict(good2, dx=0.0)) == gpe2p.EINVAL
    assert call(dict(good2, dim=4)) == gpe2p.EINVAL
    big = dict(inputs.base_params(3, 1024, 1024, 65), precision=32)  # 68.2M cells
    assert call(big) == gpe2p.EINVAL
    q = gpe2p.params(good2)
    q.bc[1] = 5
    assert f(ctypes.byref(q), fake, fake, fake, None, fake, None, 8, out, None) == gpe2p.EINVAL
    # well formed: it gets as far as the device lookup
    assert call(good2, w=None) == gpe2p.ECUDA
    assert call(good3) == gpe2p.ECUDA


def test_measurement_fault_and_network_calls_validate_on_the_host(lib):
    """The rate probes, the fault switches and the network calls refuse bad
    arguments before they touch a device, so the refusals hold without one."""
    out = ctypes.c_double()
    # gpe2p_mma_rate: N in {32, 64, 128, 256}, 1, 2 or 4 issuers, N x issuers <= 512 TMEM columns
    assert lib.gpe2p_mma_rate(48, 1, ctypes.byref(out), None) == gpe2p.EINVAL
    assert lib.gpe2p_mma_rate(64, 3, ctypes.byref(out), None) == gpe2p.EINVAL
    assert lib.gpe2p_mma_rate(256, 4, ctypes.byref(out), None) == gpe2p.EINVAL
    assert lib.gpe2p_mma_rate(128, 2, None, None) == gpe2p.EINVAL
    # gpe2p_fma_rate: precision 32 or 64, an output
    assert lib.gpe2p_fma_rate(16, ctypes.byref(out), None, None) == gpe2p.EINVAL
    assert lib.gpe2p_fma_rate(64, None, None, None) == gpe2p.EINVAL
    # fault switches without a handle
    assert lib.gpe2p_set_fault_injection(None, gpe2p.FAULT_LOSE_COPY, 1) == gpe2p.EINVAL
    assert lib.gpe2p_net_fault(None, gpe2p.FAULT_LOSE_COPY, 1) == gpe2p.EINVAL
    # network calls without a handle
    assert lib.gpe2p_net_sync(None) == gpe2p.EINVAL
    assert lib.gpe2p_net_set_backend(None, 1) == gpe2p.EINVAL
    assert lib.gpe2p_net_forward(None, None, None, 1) == gpe2p.EINVAL
    assert lib.gpe2p_net_gradients(None, None, None, 1, None, None) == gpe2p.EINVAL
    assert lib.gpe2p_net_train_step(None, None, None, 1, 1e-3, None) == gpe2p.EINVAL
    # gpe2p_net_create: each shape rule refused with its reason, and no handle left behind
    h = ctypes.c_void_p(1)

    def create(levels=4, ch=(32, 64, 128, 256), in_ch=4, out_ch=4, H=64, W=64, B=2, out=True):
        arr = (ctypes.c_int * max(len(ch), 1))(*ch)
        return lib.gpe2p_net_create(levels, arr, in_ch, out_ch, H, W, B, 0, None,
                                    ctypes.byref(h) if out else None)

    assert create(out=False) == gpe2p.EINVAL
    for kw, why in ((dict(levels=0), b"levels"), (dict(levels=7, ch=(32,) * 7), b"levels"),
                    (dict(ch=(32, 64, 120, 256)), b"channels"), (dict(ch=(8, 64, 128, 256)), b"channels"),
                    (dict(in_ch=0), b"channels"), (dict(out_ch=17), b"channels"),
                    (dict(H=60), b"multiples"), (dict(W=4), b"multiples"),
                    (dict(B=0), b"max_batch"), (dict(B=1 << 20, H=256, W=256), b"max_batch")):
        assert create(**kw) == gpe2p.EINVAL, kw
        assert h.value is None, kw
        assert why in lib.gpe2p_net_last_error(None), kw
        h = ctypes.c_void_p(1)
