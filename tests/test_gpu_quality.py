"""Device-side quality measure and the measured FP32 peak.

ashrt_quality_db (ch. 4, Eqs ch4_Qpd and ch4_Qr) against the oracle's
irls.q_db on random gathers, including a ragged length, exact
reconstructions (+inf) and all-zero reference gathers (NaN); ashrt_fp32_peak
against the device's SM count and the FP32 lane count per SM.
"""
import math

import numpy as np
import pytest

from oracle import irls

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("B,n", [(5, 64 * 256), (3, 1001), (1, 7)])
def test_quality_matches_oracle(lib, B, n):
    import torch
    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(B * n)
    o = rng.standard_normal((B, n)).astype(np.float32)
    t = (o + rng.uniform(0.01, 1.0, (B, 1)) * rng.standard_normal((B, n))).astype(np.float32)
    sums = torch.empty((B, 2), dtype=torch.float64, device=dev)
    q = ashrt.quality_db(torch.from_numpy(o).to(dev), torch.from_numpy(t).to(dev), sums)
    for b in range(B):
        assert abs(q[b] - irls.q_db(o[b], t[b])) <= 1e-9
    s = sums.cpu().numpy()
    np.testing.assert_allclose(s[:, 0], (o.astype(np.float64) ** 2).sum(1), rtol=1e-12)


def test_quality_special_cases(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda:0")
    o = torch.randn((3, 50), device=dev)
    o[2] = 0.0
    t = o.clone()
    t[1] *= 0.9                       # 20 dB exactly
    sums = torch.empty((3, 2), dtype=torch.float64, device=dev)
    q = ashrt.quality_db(o, t, sums)
    assert q[0] == math.inf and abs(q[1] - 20.0) < 1e-5 and math.isnan(q[2])


def test_fp32_peak_is_plausible(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    tf, sms = ashrt.fp32_peak(iters=2000, reps=2)
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    # 128 FP32 lanes x 2 flops per SM per clock, clocks between 0.5 and 2.2 GHz
    assert sms * 128 * 2 * 0.5e9 / 1e12 < tf < sms * 128 * 2 * 2.2e9 / 1e12
