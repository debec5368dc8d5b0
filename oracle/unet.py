"""Plain numpy FP64 reference of the surrogate network (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU legs may load it;
the product library never does.

The network is the one the C ABI (gpe2p_net_*) documents: a U-Net of L levels
on a periodic grid.  Encoder level l: [2x2 average pooling if l > 0], conv3x3
+ SiLU, conv3x3 + SiLU.  Decoder level l = L-2 .. 0: nearest 2x upsampling,
conv3x3 + SiLU, concatenation [up, skip], conv3x3 + SiLU, conv3x3 + SiLU.
Head: 1x1 convolution.  The input is zero-padded to 16 channels.  Loss: mean
squared error.  Adam with bias correction.  Tensors are NHWC float64; the
flat parameter layout is the library's: per convolution (encoder 0..L-1 a,
b; decoder L-2..0 up, a, b) weights [cout][tap][cin] with
tap = 3(dy+1) + (dx+1), then bias [cout]; then head weights [out][c0] and
bias [out].  Everything is written out with numpy primitives and explicit
loops over the nine taps; backward passes are the adjoints, derived by hand.

With bf16=True the FP64 arithmetic is kept but every tensor the network
stores in BF16 is rounded to BF16 (nearest, ties to even, through FP32) where
it is stored: the padded input, each convolution's pre-activation z (kept for
the backward pass) and its output SiLU(z) (SiLU of the unrounded z), the
pooled tensors, and in the backward pass the gradient of every stored
activation: the head's input gradient, dz = dy SiLU'(z) of each convolution,
each convolution's input gradient, the sum of the four children of an
upsampled pixel and the encoder gradient after the pooled gradient is added.
Weights and biases are given already rounded by the caller.  What remains
between this and a BF16/FP32 implementation is the accumulation (FP64 here)
and the rounding of a stored value whose FP32 and FP64 sums fall on the two
sides of a BF16 rounding boundary.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def layer_shapes(levels, channels, in_ch, out_ch):
    """[(name, cin, cout, taps)] in parameter order, and the head (cin, cout)."""
    convs = []
    for l in range(levels):
        convs.append((f"enc{l}a", 16 if l == 0 else channels[l - 1], channels[l], 9))
        convs.append((f"enc{l}b", channels[l], channels[l], 9))
    for l in range(levels - 2, -1, -1):
        convs.append((f"up{l}", channels[l + 1], channels[l], 9))
        convs.append((f"dec{l}a", 2 * channels[l], channels[l], 9))
        convs.append((f"dec{l}b", channels[l], channels[l], 9))
    return convs, (channels[0], out_ch)


def unpack(params, levels, channels, in_ch, out_ch):
    convs, (hc, ho) = layer_shapes(levels, channels, in_ch, out_ch)
    p = {}
    o = 0
    for name, cin, cout, taps in convs:
        n = cout * taps * cin
        p[name + ".w"] = params[o:o + n].reshape(cout, taps, cin)
        o += n
        p[name + ".b"] = params[o:o + cout]
        o += cout
    p["head.w"] = params[o:o + ho * hc].reshape(ho, hc)
    o += ho * hc
    p["head.b"] = params[o:o + ho]
    o += ho
    assert o == params.size
    return p


def pack(grads, levels, channels, in_ch, out_ch):
    convs, _ = layer_shapes(levels, channels, in_ch, out_ch)
    parts = []
    for name, *_ in convs:
        parts += [grads[name + ".w"].ravel(), grads[name + ".b"].ravel()]
    parts += [grads["head.w"].ravel(), grads["head.b"].ravel()]
    return np.concatenate(parts)


def round_bf16(a):
    """Round to the nearest BF16 value (8 significant bits, ties to even),
    through FP32 as a BF16/FP32 implementation holds the value first."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _same(a):
    return a


def shift(x, dy, dx):
    """s[b, y, x] = x[b, y + dy, x + dx] on the periodic grid."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv3x3(x, w, b):
    out = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dy, dx) in enumerate(TAPS):
        out += np.einsum("bhwc,oc->bhwo", shift(x, dy, dx), w[:, t, :])
    return out + b


def conv3x3_backward(x, w, dz):
    """(dx, dw, db) of z = conv3x3(x, w, b) for the output gradient dz."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (dy, dx_) in enumerate(TAPS):
        dw[:, t, :] = np.einsum("bhwc,bhwo->oc", shift(x, dy, dx_), dz)
        dx += shift(np.einsum("bhwo,oc->bhwc", dz, w[:, t, :]), -dy, -dx_)
    return dx, dw, dz.sum(axis=(0, 1, 2))


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def upsample(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample_backward(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(params, x, levels, channels, in_ch, out_ch, keep=False, bf16=False):
    """Network output for x [B, H, W, in_ch]; with keep=True also the saved
    tensors the backward pass needs; bf16=True rounds the stored tensors to
    BF16 (module docstring)."""
    r = round_bf16 if bf16 else _same
    p = unpack(params, levels, channels, in_ch, out_ch)
    B, H, W, _ = x.shape
    x16 = np.zeros((B, H, W, 16))
    x16[..., :in_ch] = r(x)
    saved = {"x16": x16}
    cur = x16
    enc = []
    for l in range(levels):
        if l > 0:
            cur = r(pool(enc[l - 1]))
            saved[f"pool{l - 1}"] = cur
        za = conv3x3(cur, p[f"enc{l}a.w"], p[f"enc{l}a.b"])
        a = r(silu(za))
        zb = conv3x3(a, p[f"enc{l}b.w"], p[f"enc{l}b.b"])
        e = r(silu(zb))
        saved.update({f"enc{l}a.in": cur, f"enc{l}a.z": r(za), f"enc{l}b.in": a, f"enc{l}b.z": r(zb)})
        enc.append(e)
    d = enc[-1]
    for l in range(levels - 2, -1, -1):
        u = upsample(d)
        zu = conv3x3(u, p[f"up{l}.w"], p[f"up{l}.b"])
        cat = np.concatenate([r(silu(zu)), enc[l]], axis=-1)
        za = conv3x3(cat, p[f"dec{l}a.w"], p[f"dec{l}a.b"])
        a = r(silu(za))
        zb = conv3x3(a, p[f"dec{l}b.w"], p[f"dec{l}b.b"])
        d = r(silu(zb))
        saved.update({f"up{l}.in": u, f"up{l}.z": r(zu), f"dec{l}a.in": cat, f"dec{l}a.z": r(za),
                      f"dec{l}b.in": a, f"dec{l}b.z": r(zb)})
    y = np.einsum("bhwc,oc->bhwo", d, p["head.w"]) + p["head.b"]
    saved["head.in"] = d
    return (y, saved) if keep else y


def loss_and_gradient(params, x, t, levels, channels, in_ch, out_ch, bf16=False):
    """Mean squared error of net(x) against t and its gradient (flat layout);
    bf16=True rounds the stored tensors and gradients to BF16 (module
    docstring)."""
    r = round_bf16 if bf16 else _same
    p = unpack(params, levels, channels, in_ch, out_ch)
    y, s = forward(params, x, levels, channels, in_ch, out_ch, keep=True, bf16=bf16)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    dy = 2.0 * (y - t) / n
    g = {}
    g["head.w"] = np.einsum("bhwc,bhwo->oc", s["head.in"], dy)
    g["head.b"] = dy.sum(axis=(0, 1, 2))
    dd = r(np.einsum("bhwo,oc->bhwc", dy, p["head.w"]))

    def layer_back(name, dout):
        dz = r(dout * dsilu(s[name + ".z"]))
        dx, dw, db = conv3x3_backward(s[name + ".in"], p[name + ".w"], dz)
        g[name + ".w"], g[name + ".b"] = dw, db
        return r(dx)

    denc = [None] * levels
    dpool_to_enc = None
    # decoder, from the output inwards
    for l in range(0, levels - 1):
        da = layer_back(f"dec{l}b", dd)
        dcat = layer_back(f"dec{l}a", da)
        c = channels[l]
        denc[l] = dcat[..., c:]
        du = layer_back(f"up{l}", dcat[..., :c])
        dd = r(upsample_backward(du))
    denc_last = dd
    for l in range(levels - 1, -1, -1):
        de = denc_last if l == levels - 1 else r(denc[l] + dpool_to_enc)
        da = layer_back(f"enc{l}b", de)
        dinp = layer_back(f"enc{l}a", da)
        if l > 0:
            dpool_to_enc = pool_backward(dinp)
    return loss, pack(g, levels, channels, in_ch, out_ch)


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (returns new w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
