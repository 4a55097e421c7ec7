"""Autotuner: every kernel variant computes the same operator (parity with
the FP64 oracle for each), the tuner picks one of them and caches it."""
import json
import os

import numpy as np
import pytest

from oracle import stolt

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_every_variant_matches_oracle(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, B = 300, 100, [1500.0, 2600.0], 3      # Nt 1024, Nx 256: all variants apply
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, wavelet_peak_hz=20.0)
    g = stolt.Geometry(nt, nx, DT, DX, v, wavelet_peak_hz=20.0)
    rng = np.random.default_rng(31)
    m = rng.standard_normal((B,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((B,) + g.data_shape).astype(np.float32)
    ref_d = stolt.forward_batch(g, m)
    ref_m = stolt.adjoint_batch(g, d)
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    for minb in (1, 2, 3, 4, 5, 6, 7, 8, 9):
        for cols in (8, 16):
            plan.set_variant(minb, cols)
            od, om = torch.empty_like(dd), torch.empty_like(md)
            plan.forward(md, od, batch=B)
            plan.adjoint(dd, om, batch=B)
            torch.cuda.synchronize()
            assert _rel(od.cpu().numpy(), ref_d) <= 1e-4, (minb, cols)
            assert _rel(om.cpu().numpy(), ref_m) <= 1e-4, (minb, cols)
    plan.close()


def test_autotune_choice_and_cache(lib, tmp_path):
    from paper_1711_10214_gb300 import ashrt
    plan = ashrt.Plan(300, 100, DT, DX, [1500.0, 2600.0], max_batch=4)
    cache = str(tmp_path / "tune.jsonl")
    mb, cols = plan.autotune(batch=4, cache_path=cache)
    assert mb in range(1, 10) and cols in (8, 16)
    lines = [json.loads(x) for x in open(cache)]
    assert len(lines) == 1 and lines[0]["rows_minb"] == mb and lines[0]["xfft_cols"] == cols
    plan2 = ashrt.Plan(300, 100, DT, DX, [1500.0, 2600.0], max_batch=4)
    assert plan2.autotune(batch=4, cache_path=cache) == (mb, cols)
    assert len(open(cache).readlines()) == 1           # served from the cache
    plan.close()
    plan2.close()


@pytest.mark.parametrize("nt,nx,v,t0,batch,mask,kw", [
    (600, 48, [1700.0, 2600.0], None, 3, False, {}),                          # Nt 2048: 16 x 16 x 8
    (1500, 20, [2100.0], None, 2, True, {}),                                   # Nt 4096: 16 x 16 x 16
    (400, 30, [1500.0, 2300.0], [0.0, 0.05], 2, False,
     dict(wavelet_peak_hz=25.0, fmax_hz=90.0)),                               # Nt 1024, AASHRT + C
    (1024, 17, [0.0, 2500.0], None, 1, False, dict(pad_t=4)),                 # Nt 4096, v = 0, pad 4
    (700, 20, [1600.0, 2500.0], [0.0, 0.03], 1, True,
     dict(wavelet_peak_hz=25.0)),                                             # Nt 2048, AASHRT, one gather
    (600, 24, [1700.0, 2600.0], [0.0, 0.02, 0.05, 0.07, 0.11], 2, False,
     dict(wavelet_peak_hz=25.0)),                                             # Nt 2048, 5 uneven shifts
])
def test_radix16_rows_match_oracle(lib, nt, nx, v, t0, batch, mask, kw):
    """The radix-16 row kernels on every length they serve, in both CTA
    shapes (variant 5: an interleaved gather pair per CTA; variant 6: one
    gather per CTA, tables read from L2) and with the forward's accumulator in
    tensor memory (variant 9, Nt 2048; the register form on other lengths),
    with the asymptote shift, the sampling mask and an odd batch (a lone
    gather in the last pair)."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    plan = ashrt.Plan(nt, nx, DT, DX, v, t0s=t0, max_batch=batch, **kw)
    g = stolt.Geometry(nt, nx, DT, DX, v, t0s=(0.0,) if t0 is None else t0, **kw)
    rng = np.random.default_rng(77)
    m = rng.standard_normal((batch,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((batch,) + g.data_shape).astype(np.float32)
    mk = (rng.random((batch, nx)) < 0.6).astype(np.float32) if mask else None
    ref_d, ref_m = stolt.forward_batch(g, m, mk), stolt.adjoint_batch(g, d, mk)
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    mkd = torch.from_numpy(mk).to(dev) if mask else None
    for variant in (5, 6, 9):
        plan.set_variant(variant, 16)
        od, om = torch.full_like(dd, float("nan")), torch.full_like(md, float("nan"))
        plan.forward(md, od, mask=mkd, batch=batch)
        plan.adjoint(dd, om, mask=mkd, batch=batch)
        torch.cuda.synchronize()
        assert _rel(od.cpu().numpy(), ref_d) <= 1e-4, variant
        assert _rel(om.cpu().numpy(), ref_m) <= 1e-4, variant
    plan.close()


@pytest.mark.parametrize("variant", [6, 9])
def test_single_gather_rows_dot_test_and_dead_rows(lib, variant):
    """Variants 6 (single-gather rows) and 9 (tensor-memory forward
    accumulator) on the benchmark's row length (Nt 2048) with velocities fast
    enough that whole (velocity, k_x) rows lie outside the cone (variant 6
    writes their panel rows as zeros without a transform): parity with the
    oracle and the FP32 dot test <L m, d> = <m, L^T d>."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, B = 1000, 40, [1500.0, 6000.0, 9000.0], 3
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, wavelet_peak_hz=25.0)
    assert plan.Nt == 2048
    plan.set_variant(variant, 16)
    g = stolt.Geometry(nt, nx, DT, DX, v, wavelet_peak_hz=25.0)
    a = g.cone_a(9000.0)
    assert np.sum(a[: g.Nx // 2 + 1] >= g.Nt // 2) > 0       # some rows fully outside
    rng = np.random.default_rng(78)
    m = rng.standard_normal((B,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((B,) + g.data_shape).astype(np.float32)
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    od, om = torch.full_like(dd, float("nan")), torch.full_like(md, float("nan"))
    plan.forward(md, od, batch=B)
    plan.adjoint(dd, om, batch=B)
    torch.cuda.synchronize()
    Lm, LTd = od.cpu().numpy().astype(np.float64), om.cpu().numpy().astype(np.float64)
    assert _rel(Lm, stolt.forward_batch(g, m)) <= 1e-4
    assert _rel(LTd, stolt.adjoint_batch(g, d)) <= 1e-4
    dot = abs(np.vdot(Lm, d) - np.vdot(m, LTd)) / (np.linalg.norm(Lm) * np.linalg.norm(d))
    assert dot <= 1e-5
    plan.close()


def test_radix16_rejected_where_it_does_not_apply(lib):
    from paper_1711_10214_gb300 import ashrt
    plan = ashrt.Plan(100, 20, DT, DX, [2000.0])        # Nt 256
    with pytest.raises(ashrt.AshrtError):
        plan.set_variant(4, 16)
    for variant in (5, 6, 7, 8):
        with pytest.raises(ashrt.AshrtError):
            plan.set_variant(variant, 16)
    with pytest.raises(ashrt.AshrtError):
        plan.set_variant(9, 16)
    with pytest.raises(ashrt.AshrtError):
        plan.set_variant(10, 16)
    plan.close()


@pytest.mark.parametrize("nt,nx,variants", [(120, 20, (1, 2, 3)), (1000, 24, (4, 5, 6, 7, 8)),
                                            (1500, 20, (4, 9))])
def test_unpadded_time_axis_every_variant(lib, nt, nx, variants):
    """pad_t = 1: the model rows fill more than half of each time transform,
    so the forward kernels run their general first pass (with the default
    padding the upper half of the input is zero and a specialised pass skips
    it); every row-kernel form against the oracle."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    v, B = [1500.0, 2600.0], 3
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, pad_t=1, wavelet_peak_hz=20.0)
    g = stolt.Geometry(nt, nx, DT, DX, v, pad_t=1, wavelet_peak_hz=20.0)
    assert plan.Nt == g.Nt and 2 * nt > plan.Nt
    rng = np.random.default_rng(32)
    m = rng.standard_normal((B,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((B,) + g.data_shape).astype(np.float32)
    ref_d, ref_m = stolt.forward_batch(g, m), stolt.adjoint_batch(g, d)
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    for variant in variants:
        plan.set_variant(variant, 16)
        od, om = torch.full_like(dd, float("nan")), torch.full_like(md, float("nan"))
        plan.forward(md, od, batch=B)
        plan.adjoint(dd, om, batch=B)
        torch.cuda.synchronize()
        assert _rel(od.cpu().numpy(), ref_d) <= 1e-4, variant
        assert _rel(om.cpu().numpy(), ref_m) <= 1e-4, variant
    plan.close()
