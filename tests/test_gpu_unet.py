"""Warm-start U-Net kernels (forward, gradients, Adam) against the FP64
reference network of ``oracle/unet.py``.

Two references.  (1) The FP64 network with the storage rounding modelled
(weights, input and stored activations rounded to bfloat16, and the masked
output gradient of each 3x3 layer rounded to bfloat16, as the tensor-core
input- and weight-gradient kernels take it; everything else exact): the
kernels differ from it only by FP32 accumulation order and the
activations that this order pushes to the neighbouring bfloat16 value (one
bfloat16 step is 2^-8 relative; after cancellation in a 9 Cin-term sum the FP32
result can be off by ~1e-5 relative, so a few in a thousand activations land
on the other side of a rounding boundary).  Outputs and loss are held to 5e-3
relative l2; parameter gradients, whose deep layers sum over few pixels
(measured up to 0.9e-2 with 64 bottleneck pixels, 0.15e-2 with 256), to
1.5e-2.
(2) The exact FP64 network: BF16 storage costs up to 2^-9 relative per
rounding, compounded over the 15 layers, and the deep levels average over few
pixels, so outputs and loss are held to 2e-2 and gradients to 5e-2 on images
with at least 4 x 8 pixels at the bottleneck.  W = 200 leaves a ragged
128-pixel tile at every level (200, 100, 50, 25 columns).
"""
import numpy as np
import pytest

from oracle import unet

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _flat(p, specs):
    return np.concatenate([np.concatenate([p[n + ".w"].ravel(), p[n + ".b"].ravel()])
                           for n, _, _, _ in specs]).astype(np.float32)


def _unflat(v, specs):
    out, o = {}, 0
    for n, ci, co, k in specs:
        out[n + ".w"] = v[o:o + co * ci * k * k].reshape(co, ci, k, k).astype(np.float64)
        o += co * ci * k * k
        out[n + ".b"] = v[o:o + co].astype(np.float64)
        o += co
    return out


def _setup(H, W, cout, n, seed):
    rng = np.random.default_rng(seed)
    specs = unet.layer_specs(1, cout)
    p = unet.init_params(rng, 1, cout)
    for name, _, co, _ in specs:
        p[name + ".b"] = 0.05 * rng.standard_normal(co)
    p = _unflat(_flat(p, specs), specs)          # the FP32 values the GPU starts from
    x = rng.standard_normal((n, H, W)).astype(np.float32) * 3.0
    return specs, p, x, rng


def _normalised(x):
    x64 = x.astype(np.float64)
    rms = np.sqrt(np.mean(x64 * x64, axis=(1, 2)))
    return x64 / rms[:, None, None], rms


Q = unet.bf16_round


@pytest.mark.parametrize("H,W,n,cout", [(16, 32, 2, 5), (24, 200, 2, 5), (16, 64, 1, 60)])
def test_forward_matches_fp64_network(lib, H, W, n, cout):
    """cout 5 and the hidden layers run on the tcgen05 kernel; a 60-channel
    head (a 64-wide tile) on the mma.sync kernel."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    specs, p, x, _ = _setup(H, W, cout, n, 31)
    net = ashrt.UNet(H, W, cout, max_batch=n, params=_flat(p, specs))
    assert net.n_params == sum(co * ci * k * k + co for _, ci, co, k in specs)
    dev = torch.device("cuda:0")
    xg = torch.from_numpy(x).to(dev)
    y = torch.empty((n, cout, H, W), device=dev)
    net.forward(xg, y)
    torch.cuda.synchronize()
    xn, rms = _normalised(x)
    yo, _ = unet.forward(p, xn[:, None], cout)
    yq, _ = unet.forward(p, xn[:, None], cout, rnd=Q)
    assert _rel(y.cpu().numpy(), yq) <= 5e-3, _rel(y.cpu().numpy(), yq)
    assert _rel(y.cpu().numpy(), yo) <= 2e-2, _rel(y.cpu().numpy(), yo)
    # outputs in input units for p = 1: panels x rms, weights exp(y) rms^-1/2
    y2 = torch.empty_like(y)
    net.forward(xg, y2, rescale=True, p=1.0)
    torch.cuda.synchronize()
    y2 = y2.cpu().numpy()
    exp_pan = yo[:, :-1] * rms[:, None, None, None]
    exp_w = np.exp(yo[:, -1]) / np.sqrt(rms)[:, None, None]
    assert _rel(y2[:, :-1], exp_pan) <= 2e-2
    assert _rel(y2[:, -1], exp_w) <= 2e-2
    net.close()


@pytest.mark.parametrize("H,W,n", [(32, 64, 2), (24, 200, 2)])
def test_gradients_match_fp64_backward(lib, H, W, n):
    import torch
    from paper_1711_10214_gb300 import ashrt
    cout = 5
    specs, p, x, rng = _setup(H, W, cout, n, 32)
    t = rng.standard_normal((n, cout, H, W)).astype(np.float32)
    lam = np.array([1.0, 1.0, 0.5, 2.0, 0.25], np.float32)
    net = ashrt.UNet(H, W, cout, max_batch=n, params=_flat(p, specs))
    dev = torch.device("cuda:0")
    loss = net.train_step(torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev), lr=0.0,
                          channel_weight=lam)
    g_gpu = _unflat(net.grads(), specs)
    xn, _ = _normalised(x)
    yo, cache = unet.forward(p, xn[:, None], cout)
    lo, gy = unet.mse_loss(yo, t.astype(np.float64), lam)
    go = unet.backward(p, cache, gy)
    yq, cq = unet.forward(p, xn[:, None], cout, rnd=Q)
    lq, gyq = unet.mse_loss(yq, t.astype(np.float64), lam)
    gq = unet.backward(p, cq, gyq, rnd=Q, rnd_g=Q)
    assert abs(loss - lq) <= 5e-3 * lq, (loss, lq)
    assert abs(loss - lo) <= 2e-2 * lo, (loss, lo)
    for name, _, _, _ in specs:
        for s in (".w", ".b"):
            k = name + s
            assert _rel(g_gpu[k], gq[k]) <= 1.5e-2, (k, _rel(g_gpu[k], gq[k]))
            assert _rel(g_gpu[k], go[k]) <= 5e-2, (k, _rel(g_gpu[k], go[k]))
    # lr = 0 leaves the parameters unchanged
    np.testing.assert_array_equal(net.params(), _flat(p, specs))
    net.close()


def test_adam_first_step_and_descent(lib):
    """Adam's first bias-corrected step is lr * g / (|g| + eps): every
    parameter whose FP64 gradient is clearly nonzero moves by lr against the
    sign of that gradient; repeated steps on one pair lower the loss."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    H, W, n, cout, lr = 32, 64, 2, 3, 1e-3
    specs, p, x, rng = _setup(H, W, cout, n, 33)
    t = rng.standard_normal((n, cout, H, W)).astype(np.float32)
    p0 = _flat(p, specs)
    net = ashrt.UNet(H, W, cout, max_batch=n, params=p0)
    dev = torch.device("cuda:0")
    xg, tg = torch.from_numpy(x).to(dev), torch.from_numpy(t).to(dev)
    l0 = net.train_step(xg, tg, lr=lr)
    step = (net.params() - p0).astype(np.float64)
    xn, _ = _normalised(x)
    yo, cache = unet.forward(p, xn[:, None], cout)
    _, gy = unet.mse_loss(yo, t.astype(np.float64))
    go = unet.backward(p, cache, gy)
    gflat = np.concatenate([np.concatenate([go[nm + ".w"].ravel(), go[nm + ".b"].ravel()])
                            for nm, _, _, _ in specs])
    big = np.abs(gflat) > 0.2 * np.abs(gflat).mean()
    assert big.mean() > 0.3
    # a ReLU unit that the BF16 network rounds dead (or alive) at a deep level
    # can zero a few gradient entries, so the property holds for >= 99%
    assert np.mean(np.abs(np.abs(step[big]) - lr) <= 2e-2 * lr) > 0.99
    assert np.mean(np.sign(step[big]) == -np.sign(gflat[big])) > 0.99
    # descent on one (random-target) pair: Adam's early steps may overshoot,
    # so the check is on the last few losses
    losses = [l0] + [net.train_step(xg, tg, lr=lr) for _ in range(30)]
    assert min(losses[-5:]) < 0.85 * losses[0], losses
    net.close()


def test_bad_sizes_are_rejected(lib):
    from paper_1711_10214_gb300 import ashrt
    with pytest.raises(ashrt.AshrtError):
        ashrt.UNet(20, 32, 3)            # H not a multiple of 8
    with pytest.raises(ashrt.AshrtError):
        ashrt.UNet(16, 32, 3, params=np.zeros(10, np.float32))
