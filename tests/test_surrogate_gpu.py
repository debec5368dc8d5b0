"""The state <-> tensor calls, the network's normalisation and the learned
surrogate with its solver check.

Packing and unpacking are data movement and are checked bit for bit against
the fields the solver reports (the density channel, a product of the
material law, to FP32 rounding).  The network's input normalisation and
residual output map are checked element by element against the numpy FP64
network oracle (with the network's BF16 storage points) composed with their
definitions.  The surrogate test trains a small network
on solver trajectories of a reduced two-drop case and shows what it gains
over the method without it: its one-call phase-field error is well below the
error of leaving the state unchanged, and the controller with the solver's
periodic check, at a check tolerance calibrated on held-out problems,
reaches the final state of the plain solver within both end-of-run bars
(phase L2 2e-2, interface within one cell).  The committed network is held
to the same bars at its calibrated tolerance on the full-size problems."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import unet
from paper_2011_00814_gb300 import build, gpe2p, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


def _state(precision, seed=4, n=64):
    prm, f = inputs.two_drops(seed, n=n, precision=precision)
    rnd = inputs.random_fields(prm, seed + 1)
    for k in ("u", "v", "p"):
        f[k] = rnd[k]
    return prm, f


@pytest.mark.parametrize("precision", [32, 64])
def test_pack_matches_fields(precision):
    import torch
    prm, f = _state(precision)
    mean = [0.1, -0.01, 0.02, 0.003, 0.5]
    scale = [0.9, 0.05, 0.04, 0.01, 0.3]
    with gpe2p.Solver(prm) as s:
        s.init_fields(f)
        t = torch.empty((64, 64, 5), dtype=torch.float32, device="cuda")
        s.pack(t, mean, scale)
        torch.cuda.synchronize()
        got = t.cpu().numpy()
        r = s.read_fields()
    ft = np.float32 if precision == 32 else np.float64
    for c, k in enumerate(("phi", "u", "v", "p")):
        want = (r[k].astype(ft).astype(np.float32) - np.float32(mean[c])) / np.float32(scale[c])
        assert np.array_equal(got[..., c], want.astype(np.float32)), k
    rho = 0.5 * ((1.0 + r["phi"]) + prm["rhoG"] * (1.0 - r["phi"]))
    assert np.max(np.abs(got[..., 4] - (rho - mean[4]) / scale[4])) < 1e-5


def test_unpack_round_trip_and_mu():
    import torch
    prm, f = _state(32)
    t = torch.empty((64, 64, 5), dtype=torch.float32, device="cuda")
    with gpe2p.Solver(prm) as a, gpe2p.Solver(prm) as b:
        # the same accumulation policy on both (the automatic switch follows the
        # drift since gpe2p_init_fields, which only `a` has)
        a.set_phi_accumulation(gpe2p.PHI_ACC_FP32)
        b.set_phi_accumulation(gpe2p.PHI_ACC_FP32)
        a.init_fields(f)
        a.advance(5)
        a.pack(t)
        torch.cuda.synchronize()
        b.unpack(t)
        ra, rb = a.read_fields(), b.read_fields()
        for k in ("phi", "u", "v", "p", "mu"):
            assert np.array_equal(ra[k], rb[k]), k
        # the unpacked problem steps on exactly as the original
        a.advance(3)
        b.advance(3)
        ra, rb = a.read_fields(), b.read_fields()
        for k in ("phi", "u", "v", "p"):
            assert np.array_equal(ra[k], rb[k]), k


def test_distance_sums():
    import torch
    prm, f = _state(64)
    prm2, f2 = _state(64, seed=11)
    t = torch.empty((64, 64, 4), dtype=torch.float32, device="cuda")
    with gpe2p.Solver(prm) as a, gpe2p.Solver(prm) as b:
        a.init_fields(f)
        b.init_fields(f2)
        b.pack(t)
        d = a.distance(t)
        torch.cuda.synchronize()
        tv = t.cpu().numpy().astype(np.float64)
        r = a.read_fields()
    for c, k in enumerate(("phi", "u", "v", "p")):
        assert math.isclose(d[2 * c], float(np.sum((r[k] - tv[..., c]) ** 2)), rel_tol=1e-12), k
        assert math.isclose(d[2 * c + 1], float(np.sum(r[k] ** 2)), rel_tol=1e-12), k


def test_batch_pack_equals_single():
    import torch
    cases = [_state(32, seed=s) for s in (1, 2, 3)]
    tb = torch.empty((3, 64, 64, 5), dtype=torch.float32, device="cuda")
    ts = torch.empty_like(tb)
    with gpe2p.Batch([p for p, _ in cases]) as b:
        for k, (_, f) in enumerate(cases):
            b.init_instance(k, f)
        b.advance(4)
        for k in range(3):
            b.pack(k, tb[k])
        torch.cuda.synchronize()
        for k, (p, f) in enumerate(cases):
            with gpe2p.Solver(p) as s:
                s.init_fields(f)
                s.advance(4)
                s.pack(ts[k])
                torch.cuda.synchronize()
        assert torch.equal(tb, ts)
        # unpack into an instance and read it back
        b.unpack(1, ts[2])
        torch.cuda.synchronize()
        r = b.read_instance(1)
    assert np.array_equal(r["phi"].astype(np.float32), ts[2, ..., 0].cpu().numpy())


def _host_interface_distance(phi_a, phi_b, bc):
    """The interface displacement measure written out on the host: central
    differences of phi_b with periodic wrap or mirrored ghosts per axis."""
    pad = [(1, 1), (1, 1)]
    mode_y = "wrap" if bc[1] == "periodic" else "symmetric"
    mode_x = "wrap" if bc[0] == "periodic" else "symmetric"
    e = np.pad(phi_b, [(1, 1), (0, 0)], mode=mode_y)
    e = np.pad(e, [(0, 0), (1, 1)], mode=mode_x)
    gx = 0.5 * (e[1:-1, 2:] - e[1:-1, :-2])
    gy = 0.5 * (e[2:, 1:-1] - e[:-2, 1:-1])
    g = np.sqrt(gx ** 2 + gy ** 2)
    d = np.abs(phi_a - phi_b)
    band = np.abs(phi_b) < 0.5
    return [float((d[band] / np.maximum(g[band], 1e-12)).max()), float(d.sum() / g.sum()), float(band.sum())]


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("noslip", "freeslip")])
def test_interface_distance_matches_host(bc):
    """gpe2p_interface_distance against the same measure on the host, for a
    tensor whose phi channel is the state's interface moved by a fraction of
    a cell; periodic and walled boxes (the gradient's ghost rules)."""
    import torch
    from paper_2011_00814_gb300 import surrogate as S
    prm, f = inputs.two_drops(7, n=64)
    prm = dict(prm, bc=bc + ("periodic",), precision=32)
    with gpe2p.Solver(prm) as s:
        s.init_fields(f)
        t = torch.empty((64, 64, 5), dtype=torch.float32, device="cuda")
        s.pack(t)
        phi_b = s.read_fields()["phi"]
        moved = np.roll(f["phi"], 1, axis=1) * 0.3 + f["phi"] * 0.7
        t[..., 0] = torch.from_numpy(moved.astype(np.float32)).cuda()
        got = s.interface_distance(t)
        want = _host_interface_distance(t[..., 0].double().cpu().numpy(), phi_b, bc)
        assert got[2] == want[2]
        assert abs(got[0] - want[0]) <= 1e-9 * want[0] and abs(got[1] - want[1]) <= 1e-9 * want[1], (got, want)
        assert 0.1 < got[0] < 3.0
        if bc[0] == "periodic":
            mean, mx = S.interface_error(t[..., 0].double().cpu().numpy(), phi_b)
            assert abs(got[0] - mx) <= 1e-9 * mx and abs(got[1] - mean) <= 1e-9 * mean


def test_net_normalisation_matches_oracle():
    import torch
    L, CH, C, H, W, B = 2, [16, 32], 5, 16, 16, 2
    net = gpe2p.Net(L, CH, C, C, H, W, B, seed=3)
    rng = np.random.default_rng(2)
    p = net.get_params()
    convs, (hc, ho) = unet.layer_shapes(L, CH, C, C)
    nh = ho * hc + ho
    p[-nh:] = rng.normal(size=nh).astype(np.float32) * 0.3
    # weights exactly representable in BF16 so that only activations round
    p = (p.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)
    net.set_params(p)
    mean = rng.normal(size=C).astype(np.float32)
    sc = rng.uniform(0.5, 2.0, size=C).astype(np.float32)
    osc = rng.uniform(0.01, 0.1, size=C).astype(np.float32)
    net.set_normalization(mean, sc, osc, residual=True)
    x = rng.normal(size=(B, H, W, C)).astype(np.float32)
    tg = x + osc * rng.normal(size=(B, H, W, C)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(tg).cuda()
    y = torch.empty_like(xd)
    net.forward(xd, y, B)
    loss, g = net.gradients(xd, td, B)
    torch.cuda.synchronize()
    # the oracle with the network's BF16 storage points (tests/test_net_gpu.py
    # states the bound: max |a - b| <= 4 x 2^-8 max |b| per compared tensor)
    xn = (x.astype(np.float64) - mean) / sc
    h = unet.forward(p.astype(np.float64), xn, L, CH, C, C, bf16=True)
    ref = x + osc * h
    dev = y.cpu().numpy()
    bound = 4.0 * 2.0 ** -8
    assert np.max(np.abs((dev - ref) / osc)) <= bound * np.max(np.abs(h))
    lref, gref = unet.loss_and_gradient(p.astype(np.float64), xn, (tg - x) / osc, L, CH, C, C, bf16=True)
    assert abs(loss - lref) < 1e-3 * lref
    o = 0
    for name, cin, cout, taps in convs:
        for n_ in (cout * taps * cin, cout):
            sl = slice(o, o + n_)
            assert np.max(np.abs(g[sl] - gref[sl])) <= bound * np.max(np.abs(gref[sl])), name
            o += n_
    assert np.max(np.abs(g[o:] - gref[o:])) <= bound * np.max(np.abs(gref[o:]))
    net.close()


def test_trained_surrogate_gains_over_persistence_and_passes_checks():
    """Reduced case: 64 x 64 box, K = 16 steps per call, a 3-level net."""
    import torch
    from paper_2011_00814_gb300 import surrogate as S
    n, K = 64, 16
    train_cases = [inputs.two_drops(s, n=n) for s in range(24)]
    test_cases = [inputs.two_drops(1000 + s, n=n) for s in range(4)]
    D, _ = S.generate(train_cases, snapshots=8, K=K)
    Dt, _ = S.generate(test_cases, snapshots=8, K=K)
    sur = S.Surrogate(n=n, K=K, levels=3, channels=(16, 32, 64), max_batch=8, seed=1)
    sur.set_stats(*S.dataset_stats(D, sample=32))
    hist = S.train(sur, D, steps=1500, batch=8, lr=2e-3, log_every=250)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    errs = S.one_call_errors(sur, Dt, [(t, k) for t in range(4) for k in range(8)])
    net_err = float(np.mean([a for a, _ in errs]))
    pers_err = float(np.mean([b for _, b in errs]))
    assert net_err < 0.5 * pers_err, (net_err, pers_err)
    # the check tolerance calibrated on two held-out problems, then both
    # end-of-run bars (phi L2 and the interface within one cell) on two others
    cal = S.calibrate_tolerance(sur, test_cases[2:4], calls=16)
    assert cal["tol_disp"] is not None, cal
    sur.check_tol_disp = cal["tol_disp"]
    for prm, f in test_cases[:2]:
        res = S.compare_to_solver(sur, prm, f, calls=16)
        assert res["stats"]["net_calls"] >= 8
        assert res["phi_l2"] <= S.BAR_PHI_L2, res
        assert res["interface_max"] <= S.BAR_INTERFACE, res
        assert res["meets_bars"]
    sur.close()
    del D, Dt
    torch.cuda.empty_cache()


def test_committed_surrogate_meets_both_bars_at_its_calibrated_tolerance():
    """The committed network (256 x 256, K = 64) at the check tolerance
    calibrated on held-out problems (the calibration file beside the
    weights): over 64 calls (4096 steps) on two evaluation problems that
    neither training nor calibration saw, the phase field ends within both
    bars of the solver's, and the controller reaches it faster than the
    plain solver."""
    import os

    from paper_2011_00814_gb300 import surrogate as S
    path = os.path.join(os.path.dirname(S.__file__), "data", "unet_two_drops_256.npz")
    sur = S.Surrogate.load(path, max_batch=1)
    assert sur.calibration is not None and sur.calibration["tol_disp"] is not None
    assert sur.check_tol == sur.calibration["tol"] == S.BAR_PHI_L2
    assert sur.check_tol_disp == sur.calibration["tol_disp"]
    lo, hi = sur.calibration["seeds"]
    for c in (0, 1):
        seed = 50000 + c
        assert not lo <= seed <= hi
        prm, f = inputs.two_drops(seed)
        res = S.compare_to_solver(sur, prm, f, calls=64)
        assert res["phi_l2"] <= S.BAR_PHI_L2, res
        assert res["interface_max"] <= S.BAR_INTERFACE, res
        assert res["speedup"] > 1.0, res
    sur.close()
