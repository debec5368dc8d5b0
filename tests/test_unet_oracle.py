"""Pins of the network oracle (oracle/unet.py) against what the mathematics
fixes: the circular convolution against a brute-force loop, the adjoint
identities of pooling and upsampling, and the analytic gradient of the whole
network against central finite differences."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import unet


def test_conv3x3_matches_brute_force():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 6, 3))
    w = rng.normal(size=(4, 9, 3))
    b = rng.normal(size=4)
    got = unet.conv3x3(x, w, b)
    ref = np.zeros((2, 5, 6, 4))
    for n in range(2):
        for y in range(5):
            for xx in range(6):
                for o in range(4):
                    s = b[o]
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            t = 3 * (dy + 1) + (dx + 1)
                            for c in range(3):
                                s += x[n, (y + dy) % 5, (xx + dx) % 6, c] * w[o, t, c]
                    ref[n, y, xx, o] = s
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def test_conv3x3_backward_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 6, 4, 3))
    w = rng.normal(size=(5, 9, 3))
    dz = rng.normal(size=(2, 6, 4, 5))
    dx, dw, db = unet.conv3x3_backward(x, w, dz)
    # <conv(x), dz> is linear in x and in w
    z0 = unet.conv3x3(x, w, np.zeros(5))
    assert abs(np.sum(z0 * dz) - np.sum(x * dx)) < 1e-10
    assert abs(np.sum(z0 * dz) - np.sum(w * dw)) < 1e-10
    assert np.allclose(db, dz.sum(axis=(0, 1, 2)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 8, 6, 3))
    y = rng.normal(size=(2, 4, 3, 3))
    assert abs(np.sum(unet.pool(x) * y) - np.sum(x * unet.pool_backward(y))) < 1e-12
    assert abs(np.sum(unet.upsample(y) * x) - np.sum(y * unet.upsample_backward(x))) < 1e-12


@pytest.mark.parametrize("levels,channels", [(1, [16]), (2, [16, 32]), (3, [16, 16, 32])])
def test_gradient_matches_finite_differences(levels, channels):
    rng = np.random.default_rng(4)
    in_ch, out_ch, H, W, B = 4, 3, 8, 8, 2
    convs, (hc, ho) = unet.layer_shapes(levels, channels, in_ch, out_ch)
    parts = []
    for _, cin, cout, taps in convs:          # weights of variance 1/fan_in keep the activations O(1)
        parts += [rng.normal(size=cout * taps * cin) / np.sqrt(taps * cin), rng.normal(size=cout) * 0.1]
    parts += [rng.normal(size=ho * hc) / np.sqrt(hc), rng.normal(size=ho) * 0.1]
    p = np.concatenate(parts)
    n = p.size
    x = rng.normal(size=(B, H, W, in_ch))
    t = rng.normal(size=(B, H, W, out_ch))
    loss, g = unet.loss_and_gradient(p, x, t, levels, channels, in_ch, out_ch)
    idx = rng.choice(n, size=40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        lp, _ = unet.loss_and_gradient(p + e, x, t, levels, channels, in_ch, out_ch)
        lm, _ = unet.loss_and_gradient(p - e, x, t, levels, channels, in_ch, out_ch)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_adam_first_steps_closed_form():
    """Bias-corrected Adam: at t = 1 each weight moves by lr g / (|g| + eps);
    with a constant gradient every step moves by lr g / (|g| + eps) too,
    since both corrected moments equal g and g^2."""
    rng = np.random.default_rng(5)
    w0 = rng.normal(size=50)
    g = rng.normal(size=50)
    lr, eps = 1e-3, 1e-8
    w, m, v = unet.adam_step(w0, g, 0.0, 0.0, 1, lr, eps=eps)
    assert np.allclose(w, w0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    for t in range(2, 6):
        w_prev = w
        w, m, v = unet.adam_step(w, g, m, v, t, lr, eps=eps)
        assert np.allclose(w - w_prev, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_round_bf16_matches_the_library_conversion():
    """The oracle's BF16 rounding (nearest, ties to even, through FP32) agrees
    with torch's float32 -> bfloat16 conversion, a library routine, on random
    values, exact halfway cases, signed zeros and powers of two."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-8, 8, size=4000),
                        [0.0, -0.0, 1.0, -2.0, 2.0 ** -20, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8,
                         -(1.0 + 2.0 ** -8), 1.0 + 2.0 ** -8 + 2.0 ** -20]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = unet.round_bf16(x)
    assert np.array_equal(got, ref)
    # ties to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert unet.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert unet.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_bf16_mode_rounds_only_what_is_stored():
    """With bf16=True every saved tensor is a BF16 value, and the output and
    gradient stay within the BF16 rounding of the FP64 network (about 2^-9 per
    stored tensor over the few layers of this net), so the mode rounds where
    values are stored and nowhere else."""
    L, ch, IN, OUT = 2, [16, 32], 3, 2
    rng = np.random.default_rng(12)
    convs, _ = unet.layer_shapes(L, ch, IN, OUT)
    n = sum(co * t * ci + co for _, ci, co, t in convs) + OUT * ch[0] + OUT
    p = unet.round_bf16(rng.normal(size=n) * 0.2)
    x = rng.normal(size=(2, 8, 8, IN))
    t = rng.normal(size=(2, 8, 8, OUT))
    y64 = unet.forward(p, x, L, ch, IN, OUT)
    y16, saved = unet.forward(p, x, L, ch, IN, OUT, keep=True, bf16=True)
    for k, v in saved.items():
        assert np.array_equal(unet.round_bf16(v), v), k
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-5 < rel < 2e-2, rel
    _, g64 = unet.loss_and_gradient(p, x, t, L, ch, IN, OUT)
    _, g16 = unet.loss_and_gradient(p, x, t, L, ch, IN, OUT, bf16=True)
    relg = np.linalg.norm(g16 - g64) / np.linalg.norm(g64)
    assert 1e-5 < relg < 5e-2, relg
