"""Pins for the FP64 U-Net reference: convolution against scipy's
correlation, and the hand-derived backward against central finite
differences of the loss."""
import numpy as np
from scipy.signal import correlate

from oracle import unet

TINY = (2, 3, 4, 5)


def test_conv_is_cross_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 8, 10))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = sum(correlate(x[n, c], w[o, c], mode="same") for c in range(3)) + b[o]
            np.testing.assert_allclose(y[n, o], ref, atol=1e-12)


def test_pool_and_upsample_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 8, 8))
    y = rng.standard_normal((1, 2, 4, 4))
    assert abs(np.sum(unet.avgpool2(x) * y) - np.sum(x * unet.avgpool2_backward(y))) < 1e-12
    assert abs(np.sum(unet.up2(y) * x) - np.sum(y * unet.up2_backward(x))) < 1e-12


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = unet.init_params(rng, cin=1, cout=3, ch=TINY)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((2, 1, 16, 16))
    t = rng.standard_normal((2, 3, 16, 16))
    lam = [1.0, 0.5, 2.0]
    y, cache = unet.forward(p, x, ch=TINY)
    L, gy = unet.mse_loss(y, t, lam)
    g = unet.backward(p, cache, gy, ch=TINY)
    h = 1e-6
    for k in ("enc1a.w", "enc2b.w", "botta.b", "dec3a.w", "dec1b.b", "head.w"):
        idx = tuple(rng.integers(0, s) for s in p[k].shape)
        old = p[k][idx]
        p[k][idx] = old + h
        Lp = unet.mse_loss(unet.forward(p, x, ch=TINY)[0], t, lam)[0]
        p[k][idx] = old - h
        Lm = unet.mse_loss(unet.forward(p, x, ch=TINY)[0], t, lam)[0]
        p[k][idx] = old
        num = (Lp - Lm) / (2 * h)
        assert abs(num - g[k][idx]) <= 1e-6 * max(1.0, abs(num)), (k, num, g[k][idx])


def test_parameter_count_is_about_one_million():
    p = unet.init_params(np.random.default_rng(3))
    n = sum(v.size for v in p.values())
    assert 0.9e6 < n < 1.3e6


def test_adam_first_step_moves_by_lr():
    p = {"w": np.array([1.0, -2.0])}
    g = {"w": np.array([0.3, -5.0])}
    unet.adam_step(p, g, {}, lr=0.01)
    np.testing.assert_allclose(p["w"], [0.99, -1.99], atol=1e-7)


def test_bf16_round_matches_torch_and_ties_to_even():
    """bfloat16 rounding against torch's CPU conversion, plus the exact cases:
    representable values unchanged, halfway values to the even neighbour."""
    import torch
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-20, 20, 2000),
                        [0.0, -0.0, 1.0, -2.5, 3.0e38]])
    x32 = x.astype(np.float32)
    want = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(unet.bf16_round(x32), want)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert unet.bf16_round(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: -> 1 + 2^-6 (even)
    assert unet.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert unet.bf16_round(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    assert unet.bf16_round(1.0 + 1.5 * 2.0 ** -8) == 1.0 + 2.0 ** -7


def test_rounded_network_reduces_to_exact_on_representable_values():
    """With weights, input and activations already bfloat16 values the
    rounding model changes nothing but the activations the convolutions
    create; with rnd = identity it is the exact network."""
    rng = np.random.default_rng(6)
    ch = (4, 6, 8, 10)
    p = unet.init_params(rng, 1, 3, ch)
    x = rng.standard_normal((1, 1, 16, 16))
    y0, _ = unet.forward(p, x, 3, ch)
    y1, _ = unet.forward(p, x, 3, ch, rnd=lambda v: v)
    np.testing.assert_array_equal(y0, y1)
    y2, _ = unet.forward(p, x, 3, ch, rnd=unet.bf16_round)
    rel = np.linalg.norm(y2 - y0) / np.linalg.norm(y0)
    assert 1e-5 < rel < 3e-2


def test_gradient_rounding_hook_only_touches_the_3x3_layers():
    """rnd_g = identity reproduces the exact backward; a real rounding leaves
    the head's gradients unchanged, is exact on values that are already
    bfloat16, and perturbs the 3x3 layers' gradients only slightly."""
    rng = np.random.default_rng(7)
    ch = (4, 6, 8, 10)
    p = unet.init_params(rng, 1, 3, ch)
    x = rng.standard_normal((1, 1, 16, 16))
    y, cache = unet.forward(p, x, 3, ch)
    gy = rng.standard_normal(y.shape)
    g0 = unet.backward(p, cache, gy, ch)
    g1 = unet.backward(p, cache, gy, ch, rnd_g=lambda v: v)
    for k in g0:
        np.testing.assert_array_equal(g0[k], g1[k])
    g2 = unet.backward(p, cache, gy, ch, rnd_g=unet.bf16_round)
    for k in ("head.w", "head.b"):
        np.testing.assert_array_equal(g0[k], g2[k])
    for k in ("dec1b.w", "enc1a.w"):
        rel = np.linalg.norm(g2[k] - g0[k]) / np.linalg.norm(g0[k])
        assert 0.0 < rel < 3e-2, (k, rel)
    # a gradient made of bfloat16 values is not changed by the rounding
    gyq = unet.bf16_round(gy)
    cache_q = {k: (v[0], v[1]) for k, v in cache.items()}
    g3 = unet.backward(p, cache_q, gyq, ch, rnd_g=lambda v: v)
    np.testing.assert_array_equal(g3["head.w"], unet.backward(p, cache, gyq, ch)["head.w"])
