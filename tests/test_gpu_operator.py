"""GPU parity of the Stolt ASHRT/AASHRT operator pair against the FP64 oracle.

Relative l2 error <= 1e-4 element by element on seeded inputs (sizes that
span several FFT passes, ragged nt/nx, every radix tail), the FP32
dot-product test <= 1e-5, and sampled parity at the full 64 x 1024 x 256 x 32
benchmark configuration.
"""
import numpy as np
import pytest

from oracle import stolt
from paper_1711_10214_gb300 import synth

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5
TOL = 1e-4


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(lib, torch, nt, nx, v, t0=None, batch=1, mask=False, seed=0, **kw):
    from paper_1711_10214_gb300 import ashrt
    plan = ashrt.Plan(nt, nx, DT, DX, v, t0s=t0, max_batch=batch, **kw)
    g = stolt.Geometry(nt, nx, DT, DX, v, t0s=(0.0,) if t0 is None else t0, **kw)
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((batch,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((batch,) + g.data_shape).astype(np.float32)
    mk = (rng.random((batch, nx)) < 0.6).astype(np.float32) if mask else None
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    mkd = torch.from_numpy(mk).to(dev) if mask else None
    od, om = torch.empty_like(dd), torch.empty_like(md)
    plan.forward(md, od, mask=mkd, batch=batch)
    plan.adjoint(dd, om, mask=mkd, batch=batch)
    torch.cuda.synchronize()
    od, om = od.cpu().numpy().astype(np.float64), om.cpu().numpy().astype(np.float64)
    ref_d = stolt.forward_batch(g, m, mk)
    ref_m = stolt.adjoint_batch(g, d, mk)
    # FP32 dot test of the GPU pair itself
    dot = abs(np.vdot(od, d.astype(np.float64)) - np.vdot(m.astype(np.float64), om))
    dot /= np.linalg.norm(od) * np.linalg.norm(d)
    plan.close()
    return _rel(od, ref_d), _rel(om, ref_m), dot


@pytest.mark.parametrize("nt,nx,v,t0,batch,mask,kw", [
    (256, 64, synth.velocity_scan(1500, 3000, 8), None, 1, False, {}),          # config-1 sizes
    (50, 13, [1800.0, 2500.0], None, 2, False, {}),                              # ragged, Nt 128 Nx 32
    (100, 37, [1500.0, 2000.0, 3500.0], None, 1, True, {}),                      # mask S
    (64, 16, [0.0, 2000.0], None, 3, False, dict(pad_t=4, pad_x=1)),             # v = 0, no x pad
    (96, 24, [1500.0, 2300.0], [0.0, 0.06, 0.1], 2, False,
     dict(wavelet_peak_hz=25.0, fmax_hz=90.0)),                                  # AASHRT + C + band
    (300, 20, [2000.0], [0.035], 1, False, {}),                                  # Nt 1024, one shift
    (600, 48, [1700.0, 2600.0], None, 1, False, {}),                             # Nt 2048
])
def test_operator_parity(lib, nt, nx, v, t0, batch, mask, kw):
    import torch
    ef, ea, dot = _case(lib, torch, nt, nx, v, t0, batch, mask, **kw)
    assert ef <= TOL, ef
    assert ea <= TOL, ea
    assert dot <= 1e-5, dot


def test_every_fft_length(lib):
    """Nt from 64 to 4096 and Nx from 16 to 2048 (all radix tails 2, 4, 8)."""
    import torch
    for nt, nx, kw in [(32, 8, {}), (64, 16, {}), (1000, 9, {}), (1500, 5, {}),
                       (40, 300, {}), (40, 600, {}), (40, 1000, {})]:
        ef, ea, dot = _case(lib, torch, nt, nx, [2100.0], **kw)
        assert ef <= TOL and ea <= TOL and dot <= 1e-5, (nt, nx, ef, ea, dot)


def test_full_size_sampled_parity(lib):
    """Benchmark configuration (64 gathers, nt 1024, nx 256, 32 velocities):
    GPU dot test over the whole batch, and panel-restricted parity on one
    gather against the oracle (linearity: only two velocity panels carry
    energy, so the oracle needs only those two)."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, B = 1024, 256, 64
    v = synth.velocity_scan(1400, 3500, 32)
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B)
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev).manual_seed(5)
    m = torch.randn((B, 1, 32, nx, nt), device=dev, generator=gen)
    d = torch.randn((B, nx, nt), device=dev, generator=gen)
    od, om = torch.empty_like(d), torch.empty_like(m)
    plan.forward(m, od, batch=B)
    plan.adjoint(d, om, batch=B)
    torch.cuda.synchronize()
    lhs = torch.sum(od.double() * d.double()).item()
    rhs = torch.sum(m.double() * om.double()).item()
    assert abs(lhs - rhs) / (od.double().norm().item() * d.double().norm().item()) < 1e-5

    # one gather, energy in panels 0 and 31 only
    rng = np.random.default_rng(9)
    m1 = np.zeros((1, 1, 32, nx, nt), np.float32)
    m1[0, 0, 0] = rng.standard_normal((nx, nt))
    m1[0, 0, 31] = rng.standard_normal((nx, nt))
    d1 = rng.standard_normal((1, nx, nt)).astype(np.float32)
    mg = torch.zeros_like(m)
    mg[:1] = torch.from_numpy(m1).to(dev)
    dg = torch.zeros_like(d)
    dg[:1] = torch.from_numpy(d1).to(dev)
    plan.forward(mg, od, batch=B)
    plan.adjoint(dg, om, batch=B)
    torch.cuda.synchronize()
    g2 = stolt.Geometry(nt, nx, DT, DX, [v[0], v[31]])
    ref_d = stolt.forward(g2, m1[0][:, [0, 31]].astype(np.float64))
    ref_m = stolt.adjoint(g2, d1[0].astype(np.float64))
    assert _rel(od[0].cpu().numpy(), ref_d) <= TOL
    got = om[0, 0].cpu().numpy()[[0, 31]]
    assert _rel(got, ref_m[0]) <= TOL
    assert float(od[1:].abs().max()) == 0.0
    plan.close()
