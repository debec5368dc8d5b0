"""The state <-> tensor calls, the network's normalisation and the learned
surrogate with its solver check.

Packing and unpacking are data movement and are checked bit for bit against
the fields the solver reports (the density channel, a product of the
material law, to FP32 rounding).  The network's input normalisation and
residual output map are checked against the numpy FP64 network oracle
composed with their definitions.  The surrogate test trains a small network
on solver trajectories of a reduced two-drop case and shows what it gains
over the method without it: its one-call phase-field error is well below the
error of leaving the state unchanged, and the controller with the solver's
periodic check reaches the final state of the plain solver within the phase
L2 tolerance 2e-2."""
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
    xn = (x.astype(np.float64) - mean) / sc
    h = unet.forward(p.astype(np.float64), xn, L, CH, C, C)
    ref = x + osc * h
    dev = y.cpu().numpy()
    assert np.linalg.norm((dev - ref) / osc) / np.linalg.norm((ref - x) / osc) < 2e-2
    lref, gref = unet.loss_and_gradient(p.astype(np.float64), xn, (tg - x) / osc, L, CH, C, C)
    assert abs(loss - lref) < 2e-2 * lref
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 5e-2
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
    prm, f = test_cases[0]
    res = S.compare_to_solver(sur, prm, f, calls=16)
    assert res["stats"]["net_calls"] >= 8
    assert res["phi_l2"] <= 2e-2, res
    sur.close()
    del D, Dt
    torch.cuda.empty_cache()
