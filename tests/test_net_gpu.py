"""The surrogate network's CUDA kernels against the numpy FP64 network oracle,
for both kernel families of the 3x3 convolutions (tcgen05 with the
accumulator in tensor memory, and warp-level mma.sync).

The GPU stores weights and activations in BF16 (8 significant bits, relative
rounding 2^-9 ~ 2e-3) and accumulates in FP32.  The oracle is given the same
weights rounded to BF16, so the remaining difference is the rounding of the
activations, about 2e-3 per layer over the ~15 layers of the test network:
tolerances 2e-2 (outputs, relative L2) and 5e-2 (gradients of each layer,
relative L2) cover it with margin.  The Adam step is FP32 on both sides."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import unet
from paper_2011_00814_gb300 import build, gpe2p

pytestmark = pytest.mark.gpu

LEVELS, CHANNELS, IN, OUT, H, W, B = 3, [16, 32, 64], 4, 4, 32, 32, 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


def bf16_round(a):
    """Round float32 values to the nearest BF16 (ties to even)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def conv_weight_mask(levels, channels, in_ch, out_ch):
    """True for the entries of the flat parameters that the GPU uses in BF16
    (convolution weights; biases and the head stay FP32)."""
    convs, (hc, ho) = unet.layer_shapes(levels, channels, in_ch, out_ch)
    m = []
    for _, cin, cout, taps in convs:
        m += [np.ones(cout * taps * cin, bool), np.zeros(cout, bool)]
    m += [np.zeros(ho * hc + ho, bool)]
    return np.concatenate(m)


def layer_slices(levels, channels, in_ch, out_ch):
    convs, (hc, ho) = unet.layer_shapes(levels, channels, in_ch, out_ch)
    out, o = [], 0
    for name, cin, cout, taps in convs:
        n = cout * taps * cin + cout
        out.append((name, slice(o, o + n)))
        o += n
    out.append(("head", slice(o, o + ho * hc + ho)))
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def setup(tc=True):
    import torch
    net = gpe2p.Net(LEVELS, CHANNELS, IN, OUT, H, W, B, seed=5)
    net.set_backend(tc)
    rng = np.random.default_rng(9)
    p = net.get_params()
    # a head of order one so that the outputs are not dominated by the bias
    sl = layer_slices(LEVELS, CHANNELS, IN, OUT)[-1][1]
    p[sl] = rng.normal(size=sl.stop - sl.start).astype(np.float32) * 0.3
    net.set_params(p)
    x = rng.normal(size=(B, H, W, IN)).astype(np.float32)
    t = (rng.normal(size=(B, H, W, OUT)) * 0.5).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    mask = conv_weight_mask(LEVELS, CHANNELS, IN, OUT)
    pref = p.astype(np.float64)
    pref[mask] = bf16_round(p[mask]).astype(np.float64)
    return net, p, pref, x, t, xd, td


@pytest.mark.parametrize("tc", [True, False])
def test_forward_matches_oracle(tc):
    import torch
    net, p, pref, x, t, xd, td = setup(tc)
    y = torch.empty((B, H, W, OUT), dtype=torch.float32, device="cuda")
    net.forward(xd, y, B)
    torch.cuda.synchronize()
    ref = unet.forward(pref, x.astype(np.float64), LEVELS, CHANNELS, IN, OUT)
    assert rel(y.cpu().numpy(), ref) < 2e-2
    net.close()


@pytest.mark.parametrize("tc", [True, False])
def test_gradients_match_oracle(tc):
    net, p, pref, x, t, xd, td = setup(tc)
    loss, g = net.gradients(xd, td, B)
    lref, gref = unet.loss_and_gradient(pref, x.astype(np.float64), t.astype(np.float64), LEVELS, CHANNELS, IN, OUT)
    assert abs(loss - lref) < 2e-2 * lref
    for name, sl in layer_slices(LEVELS, CHANNELS, IN, OUT):
        assert rel(g[sl], gref[sl]) < 5e-2, (name, rel(g[sl], gref[sl]))
    net.close()


def test_adam_step_matches_oracle():
    net, p, pref, x, t, xd, td = setup()
    _, g = net.gradients(xd, td, B)
    lr = 1e-3
    net.train_step(xd, td, B, lr)
    p1 = net.get_params()
    w, _, _ = unet.adam_step(p.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, lr)
    # at t = 1 Adam moves each weight by about lr sign(g); compare where the gradient is not tiny
    big = np.abs(g) > 1e-4 * np.max(np.abs(g))
    assert np.max(np.abs(p1[big] - w[big])) < 1e-2 * lr
    net.close()


def test_training_learns_a_smooth_map():
    """A learnable target (a fixed smooth function of the input) is fitted:
    the loss falls by more than 4x in 150 Adam steps."""
    import torch
    net, p, pref, x, t, xd, td = setup()
    tl = 0.5 * xd + 0.25 * torch.roll(xd, 1, dims=1)
    l0 = net.train_step(xd, tl, B, 2e-3)
    for _ in range(150):
        l1 = net.train_step(xd, tl, B, 2e-3)
    assert l1 < 0.25 * l0, (l0, l1)
    net.close()


@pytest.mark.parametrize("shape", [(4, [32, 64, 128, 256], 64, 64, 2), (2, [16, 48], 24, 40, 3)])
def test_tcgen05_and_mma_sync_agree(shape):
    """Larger layers (N tiles of 128, several K chunks) and ragged tiles
    (24 x 40 images: 16-row tiles that overhang the image): both kernel
    families compute the same convolutions up to BF16 rounding of the
    activations."""
    import torch
    L, ch, h, w, b = shape
    net = gpe2p.Net(L, ch, IN, OUT, h, w, b, seed=7)
    rng = np.random.default_rng(3)
    p = net.get_params()
    sl = layer_slices(L, ch, IN, OUT)[-1][1]
    p[sl] = rng.normal(size=sl.stop - sl.start).astype(np.float32) * 0.3
    net.set_params(p)
    x = torch.from_numpy(rng.normal(size=(b, h, w, IN)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(size=(b, h, w, OUT)).astype(np.float32)).cuda()
    ys = []
    gs = []
    for tc in (True, False):
        net.set_backend(tc)
        y = torch.empty((b, h, w, OUT), dtype=torch.float32, device="cuda")
        net.forward(x, y, b)
        net.sync()
        ys.append(y.cpu().numpy())
        gs.append(net.gradients(x, t, b)[1])
    assert rel(ys[0], ys[1]) < 2e-2
    for name, s_ in layer_slices(L, ch, IN, OUT):
        assert rel(gs[0][s_], gs[1][s_]) < 5e-2, name
    net.close()
