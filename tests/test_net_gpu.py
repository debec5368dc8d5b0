"""The surrogate network's CUDA kernels against the numpy FP64 network oracle,
element by element, for both kernel families of the 3x3 convolutions
(tcgen05 with the accumulator in tensor memory, and warp-level mma.sync), at
the production shape (4 levels of 32-64-128-256 channels, several K chunks
and N tiles of 128) on a 64 x 64 image and on a ragged 40 x 24 image (tiles
that overhang it), and on a small 3-level net.

The GPU stores weights, activations, pre-activations and activation
gradients in BF16 (8 significant bits) and accumulates in FP32.  The oracle
runs with bf16=True: it takes the same BF16-rounded weights and rounds every
tensor the GPU stores to BF16 at the same point, accumulating in FP64.  What
remains is the accumulation order and precision (FP32 sums of up to
9 x 256 products: about 2^-24 sqrt(K) ~ 3e-6 of the summed magnitudes) and
the stored values whose FP32 and FP64 sums fall on the two sides of a BF16
rounding boundary, which then differ by one BF16 unit (2^-8 relative).  Such
flips are sparse, a few per thousand values, and a flipped input moves a
following sum by a small fraction of its own unit, so each compared value
stays within a few units of 2^-8 of the largest value it is compared with:
the bound is max |a - b| <= C 2^-8 max |b| with C = 4, for the network
output and for each layer's weight and bias gradients separately.  The tests
print the measured C.  The Adam step is FP32 on both sides."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import unet
from paper_2011_00814_gb300 import build, gpe2p

pytestmark = pytest.mark.gpu

IN, OUT = 4, 4
C_BOUND = 4.0
ULP = 2.0 ** -8
SHAPES = {
    "small": (3, [16, 32, 64], 32, 32, 2),
    "production": (4, [32, 64, 128, 256], 64, 64, 2),
    "production-ragged": (4, [32, 64, 128, 256], 40, 24, 2),
}
LEVELS, CHANNELS, H, W, B = SHAPES["small"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


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
    """[(name, weight slice, bias slice)] of the flat parameters."""
    convs, (hc, ho) = unet.layer_shapes(levels, channels, in_ch, out_ch)
    out, o = [], 0
    for name, cin, cout, taps in convs:
        nw = cout * taps * cin
        out.append((name, slice(o, o + nw), slice(o + nw, o + nw + cout)))
        o += nw + cout
    out.append(("head", slice(o, o + ho * hc), slice(o + ho * hc, o + ho * hc + ho)))
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def units(a, b):
    """max |a - b| in units of 2^-8 max |b|."""
    return float(np.max(np.abs(a - b)) / (ULP * max(float(np.max(np.abs(b))), 1e-30)))


def setup(tc=True, shape="small"):
    import torch
    L, ch, h, w, b = SHAPES[shape]
    net = gpe2p.Net(L, ch, IN, OUT, h, w, b, seed=5)
    net.set_backend(tc)
    rng = np.random.default_rng(9)
    p = net.get_params()
    # a head of order one so that the outputs are not dominated by the bias
    sl = layer_slices(L, ch, IN, OUT)[-1]
    p[sl[1]] = rng.normal(size=sl[1].stop - sl[1].start).astype(np.float32) * 0.3
    # nonzero biases, so that the bias paths are compared too
    for _, _, bs in layer_slices(L, ch, IN, OUT)[:-1]:
        p[bs] = rng.normal(size=bs.stop - bs.start).astype(np.float32) * 0.05
    net.set_params(p)
    x = rng.normal(size=(b, h, w, IN)).astype(np.float32)
    t = (rng.normal(size=(b, h, w, OUT)) * 0.5).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    mask = conv_weight_mask(L, ch, IN, OUT)
    pref = p.astype(np.float64)
    pref[mask] = unet.round_bf16(p[mask])
    return net, p, pref, x, t, xd, td


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("tc", [True, False])
def test_forward_matches_oracle_elementwise(tc, shape):
    import torch
    L, ch, h, w, b = SHAPES[shape]
    net, p, pref, x, t, xd, td = setup(tc, shape)
    y = torch.empty((b, h, w, OUT), dtype=torch.float32, device="cuda")
    net.forward(xd, y, b)
    net.sync()
    ref = unet.forward(pref, x.astype(np.float64), L, ch, IN, OUT, bf16=True)
    c = units(y.cpu().numpy(), ref)
    print(f"forward {shape} tc={tc}: C = {c:.3f}")
    assert c <= C_BOUND, c
    net.close()


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("tc", [True, False])
def test_gradients_match_oracle_elementwise(tc, shape):
    L, ch, h, w, b = SHAPES[shape]
    net, p, pref, x, t, xd, td = setup(tc, shape)
    loss, g = net.gradients(xd, td, b)
    lref, gref = unet.loss_and_gradient(pref, x.astype(np.float64), t.astype(np.float64), L, ch, IN, OUT,
                                        bf16=True)
    assert abs(loss - lref) <= 1e-3 * lref, (loss, lref)
    worst = []
    for name, ws, bs in layer_slices(L, ch, IN, OUT):
        cw, cb = units(g[ws], gref[ws]), units(g[bs], gref[bs])
        worst.append((max(cw, cb), name))
        assert cw <= C_BOUND and cb <= C_BOUND, (name, cw, cb)
    print(f"gradients {shape} tc={tc}: worst C = {max(worst)}")
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
    for name, ws, bs in layer_slices(L, ch, IN, OUT):
        assert rel(gs[0][ws], gs[1][ws]) < 5e-2, name
        assert rel(gs[0][bs], gs[1][bs]) < 5e-2, name
    net.close()
