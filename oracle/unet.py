"""FP64 reference of the warm-start U-Net (forward and hand-derived backward).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The thesis has no learned component; this network is the library's learned
warm start: it maps a pseudo-deblended gather to an initial Radon model
and initial IRLS residual weights.  Architecture (4 levels, channels ch):
  enc1: conv3x3(cin->c0) relu, conv3x3(c0->c0) relu        -> s1
  avgpool2;  enc2: (c0->c1) relu, (c1->c1) relu            -> s2
  avgpool2;  enc3: (c1->c2) relu, (c2->c2) relu            -> s3
  avgpool2;  bott: (c2->c3) relu, (c3->c3) relu
  up2 (nearest), concat s3 -> dec3: (c3+c2->c2) relu, (c2->c2) relu
  up2, concat s2 -> dec2: (c2+c1->c1) relu, (c1->c1) relu
  up2, concat s1 -> dec1: (c1+c0->c0) relu, (c0->c0) relu
  head: conv1x1(c0->cout), no activation
Convolutions are cross-correlations with zero "same" padding; tensors are
[batch][channel][height][width]; weights [cout][cin][k][k].
"""
import numpy as np

CHANNELS = (16, 48, 96, 192)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE binary32 value; rounding adds
    0x7fff plus the lowest kept bit before truncating (finite inputs only).
    The value is first rounded to binary32.
    """
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_specs(cin=1, cout=25, ch=CHANNELS):
    c0, c1, c2, c3 = ch
    return [("enc1a", cin, c0, 3), ("enc1b", c0, c0, 3),
            ("enc2a", c0, c1, 3), ("enc2b", c1, c1, 3),
            ("enc3a", c1, c2, 3), ("enc3b", c2, c2, 3),
            ("botta", c2, c3, 3), ("bottb", c3, c3, 3),
            ("dec3a", c3 + c2, c2, 3), ("dec3b", c2, c2, 3),
            ("dec2a", c2 + c1, c1, 3), ("dec2b", c1, c1, 3),
            ("dec1a", c1 + c0, c0, 3), ("dec1b", c0, c0, 3),
            ("head", c0, cout, 1)]


def init_params(rng, cin=1, cout=25, ch=CHANNELS):
    """He-normal weights, zero biases."""
    p = {}
    for name, ci, co, k in layer_specs(cin, cout, ch):
        p[name + ".w"] = rng.standard_normal((co, ci, k, k)) * np.sqrt(2.0 / (ci * k * k))
        p[name + ".b"] = np.zeros(co)
    return p


def conv(x, w, b):
    """y[n, o, i, j] = b[o] + sum_{c, u, v} w[o, c, u, v] x[n, c, i + u - r, j + v - r]."""
    k = w.shape[-1]
    r = k // 2
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (r, r), (r, r)))
    y = np.zeros((n, w.shape[0], h, wd))
    for u in range(k):
        for v in range(k):
            y += np.einsum("oc,nchw->nohw", w[:, :, u, v], xp[:, :, u:u + h, v:v + wd])
    return y + b[None, :, None, None]


def conv_backward(x, w, gy):
    """Gradients of conv(x, w, b) with respect to x, w and b."""
    k = w.shape[-1]
    r = k // 2
    n, c, h, wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (r, r), (r, r)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for u in range(k):
        for v in range(k):
            gw[:, :, u, v] = np.einsum("nohw,nchw->oc", gy, xp[:, :, u:u + h, v:v + wd])
            gxp[:, :, u:u + h, v:v + wd] += np.einsum("oc,nohw->nchw", w[:, :, u, v], gy)
    gx = gxp[:, :, r:r + h, r:r + wd]
    return gx, gw, gy.sum(axis=(0, 2, 3))


def avgpool2(x):
    n, c, h, w = x.shape
    return x.reshape(n, c, h // 2, 2, w // 2, 2).mean(axis=(3, 5))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=2), 2, axis=3) * 0.25


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up2_backward(gy):
    n, c, h, w = gy.shape
    return gy.reshape(n, c, h // 2, 2, w // 2, 2).sum(axis=(3, 5))


def forward(p, x, cout=25, ch=CHANNELS, rnd=None):
    """Returns (y, cache).

    rnd (optional, e.g. bf16_round) is applied to the weights, the input and
    every stored activation (each ReLU output and each pooled map), which
    models a network that stores them at reduced precision; None = exact.
    """
    cache = {}
    q = (lambda v: v) if rnd is None else rnd

    def cr(name, inp):
        z = conv(inp, q(p[name + ".w"]), p[name + ".b"])
        a = q(np.maximum(z, 0.0))
        cache[name] = (inp, a)
        return a

    x = q(x)
    s1 = cr("enc1b", cr("enc1a", x))
    s2 = cr("enc2b", cr("enc2a", q(avgpool2(s1))))
    s3 = cr("enc3b", cr("enc3a", q(avgpool2(s2))))
    bt = cr("bottb", cr("botta", q(avgpool2(s3))))
    d3 = cr("dec3b", cr("dec3a", np.concatenate([up2(bt), s3], axis=1)))
    d2 = cr("dec2b", cr("dec2a", np.concatenate([up2(d3), s2], axis=1)))
    d1 = cr("dec1b", cr("dec1a", np.concatenate([up2(d2), s1], axis=1)))
    y = conv(d1, q(p["head.w"]), p["head.b"])
    cache["head"] = (d1, None)
    return y, cache


def backward(p, cache, gy, ch=CHANNELS, rnd=None, rnd_g=None):
    """Gradients of sum(gy * y) with respect to every parameter.

    rnd: the rounding of the weights used in the forward pass.  rnd_g
    (optional): a rounding of the masked output gradient of each 3x3 layer,
    used for that layer's input, weight and bias gradients (the head's
    gradient is not rounded), which models a network that runs those
    products at reduced precision.  None = exact."""
    c0, c1, c2, c3 = ch
    g = {}
    q = (lambda v: v) if rnd is None else rnd
    qg = (lambda v: v) if rnd_g is None else rnd_g

    def cr_back(name, ga):
        inp, a = cache[name]
        gz = qg(ga * (a > 0.0))
        gx, gw, gb = conv_backward(inp, q(p[name + ".w"]), gz)
        g[name + ".w"], g[name + ".b"] = gw, gb
        return gx

    d1 = cache["head"][0]
    gd1, g["head.w"], g["head.b"] = conv_backward(d1, q(p["head.w"]), gy)
    gcat1 = cr_back("dec1a", cr_back("dec1b", gd1))
    gd2_up, gs1 = gcat1[:, :c1], gcat1[:, c1:]
    gcat2 = cr_back("dec2a", cr_back("dec2b", up2_backward(gd2_up)))
    gd3_up, gs2 = gcat2[:, :c2], gcat2[:, c2:]
    gcat3 = cr_back("dec3a", cr_back("dec3b", up2_backward(gd3_up)))
    gbt_up, gs3 = gcat3[:, :c3], gcat3[:, c3:]
    gp3 = cr_back("botta", cr_back("bottb", up2_backward(gbt_up)))
    gs3 = gs3 + avgpool2_backward(gp3)
    gp2 = cr_back("enc3a", cr_back("enc3b", gs3))
    gs2 = gs2 + avgpool2_backward(gp2)
    gp1 = cr_back("enc2a", cr_back("enc2b", gs2))
    gs1 = gs1 + avgpool2_backward(gp1)
    cr_back("enc1a", cr_back("enc1b", gs1))
    return g


def mse_loss(y, t, channel_weight=None):
    """L = sum_c lambda_c mean((y - t)^2); returns (L, dL/dy)."""
    n, c, h, w = y.shape
    lam = np.ones(c) if channel_weight is None else np.asarray(channel_weight, dtype=np.float64)
    e = y - t
    cnt = n * h * w
    L = float(np.sum(lam[None, :, None, None] * e * e) / cnt)
    return L, 2.0 * lam[None, :, None, None] * e / cnt


def adam_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba) of every parameter, bias-corrected."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m." + k, np.zeros_like(p[k]))
        v = state.setdefault("v." + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
