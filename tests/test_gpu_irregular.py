"""Traces at irregular positions on the GPU (ch. 6: for non-uniform spatial
sampling the trace-axis Fourier operator becomes a DFT evaluated at the trace
positions) against the FP64 oracle (oracle/stolt.py forward_irregular /
adjoint_irregular): operator parity <= 1e-4 on jittered, random, denser and
sparser trace sets with the wavelet, asymptote shifts, the trace mask and a
batch; the FP32 dot test; regular positions reproduce the regular plan; and
the robust IRLS deblend of irregularly sampled gathers against the oracle
IRLS on the oracle's irregular operator (<= 1e-3)."""
import numpy as np
import pytest

from oracle import irls, stolt

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _positions(kind, nx, nr, rng):
    if kind == "jitter":            # one trace near each apex, +-0.4 dx
        return (np.arange(nr) + rng.uniform(-0.4, 0.4, nr)) * DX
    if kind == "random":            # anywhere on the line, unsorted
        return rng.uniform(0.0, (nx - 1) * DX, nr)
    return np.arange(nr) * DX


@pytest.mark.parametrize("nt,nx,nr,kind,v,t0,kw,batch,mask", [
    (96, 24, 24, "jitter", [1500.0, 2300.0], None, dict(wavelet_peak_hz=25.0), 2, False),
    (120, 30, 45, "random", [1700.0, 2600.0], [0.0, 0.05], {}, 3, True),
    (80, 40, 13, "random", [2000.0], None, dict(fmax_hz=70.0), 1, False),
    (300, 64, 70, "jitter", [1400.0, 2100.0, 3300.0], None, dict(wavelet_peak_hz=20.0), 2, True),
])
def test_irregular_operator_parity(lib, nt, nx, nr, kind, v, t0, kw, batch, mask):
    import torch
    from paper_1711_10214_gb300 import ashrt
    rng = np.random.default_rng(nt + nr)
    x = _positions(kind, nx, nr, rng)
    plan = ashrt.Plan(nt, nx, DT, DX, v, t0s=t0, max_batch=batch, trace_x=x, **kw)
    assert plan.data_shape == (nr, nt)
    g = stolt.Geometry(nt, nx, DT, DX, v, t0s=(0.0,) if t0 is None else t0, **kw)
    m = rng.standard_normal((batch,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((batch, nr, nt)).astype(np.float32)
    mk = (rng.random((batch, nr)) < 0.7).astype(np.float32) if mask else None
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    mkd = torch.from_numpy(mk).to(dev) if mask else None
    od, om = torch.full_like(dd, float("nan")), torch.full_like(md, float("nan"))
    plan.forward(md, od, mask=mkd, batch=batch)
    plan.adjoint(dd, om, mask=mkd, batch=batch)
    torch.cuda.synchronize()
    for b in range(batch):
        mb = None if mk is None else mk[b].astype(np.float64)
        ref_d = stolt.forward_irregular(g, m[b].astype(np.float64), x, mb)
        ref_m = stolt.adjoint_irregular(g, d[b].astype(np.float64), x, mb)
        assert _rel(od[b].cpu().numpy(), ref_d) <= 1e-4, b
        assert _rel(om[b].cpu().numpy(), ref_m) <= 1e-4, b
    # FP32 dot test of the GPU pair
    Lm, LTd = od.cpu().numpy().astype(np.float64), om.cpu().numpy().astype(np.float64)
    dot = abs(np.vdot(Lm, d) - np.vdot(m, LTd)) / (np.linalg.norm(Lm) * np.linalg.norm(d))
    assert dot <= 1e-5
    plan.close()


def test_regular_positions_reproduce_the_regular_plan(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, B = 200, 48, [1600.0, 2800.0], 2
    rng = np.random.default_rng(3)
    irr = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, trace_x=np.arange(nx) * DX,
                     wavelet_peak_hz=25.0)
    reg = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, wavelet_peak_hz=25.0)
    dev = torch.device("cuda:0")
    m = torch.from_numpy(rng.standard_normal((B,) + reg.model_shape).astype(np.float32)).to(dev)
    d = torch.from_numpy(rng.standard_normal((B, nx, nt)).astype(np.float32)).to(dev)
    a, b = torch.empty_like(d), torch.empty_like(d)
    irr.forward(m, a, batch=B)
    reg.forward(m, b, batch=B)
    ma, mb = torch.empty_like(m), torch.empty_like(m)
    irr.adjoint(d, ma, batch=B)
    reg.adjoint(d, mb, batch=B)
    torch.cuda.synchronize()
    assert _rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-5
    assert _rel(ma.cpu().numpy(), mb.cpu().numpy()) <= 1e-5
    irr.close()
    reg.close()


def test_irregular_deblend_matches_oracle(lib):
    """The robust solve (ch. 4) on gathers recorded at jittered positions:
    the data-side weights, mask, median/MAD and misfit run over the nr
    recorded traces."""
    import torch
    from paper_1711_10214_gb300 import ashrt, synth
    nt, nx, nr, v, B = 80, 20, 17, [1500.0, 2400.0], 2
    rng = np.random.default_rng(4)
    x = np.sort(rng.uniform(0.0, (nx - 1) * DX, nr))
    ev = dict(tau=np.array([0.12, 0.2]), xa=np.array([60.0, 150.0]), v=np.array([1600.0, 2300.0]),
              A=np.array([1.0, -0.8]), t0=np.zeros(2))
    d = np.zeros((B, nr, nt))
    for b in range(B):
        t = np.arange(nt) * DT
        for tau, xa, vv, A in zip(ev["tau"], ev["xa"], ev["v"], ev["A"]):
            tx = np.sqrt(tau ** 2 + ((x - xa) / vv) ** 2)
            d[b] += A * synth.ricker(t[None, :] - tx[:, None], 25.0)
        d[b] += (b + 1) * 0.5 * (rng.random((nr, nt)) < 0.03) * rng.standard_normal((nr, nt))
    d = d.astype(np.float32)
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, with_solver=True, trace_x=x)
    dev = torch.device("cuda:0")
    dd = torch.from_numpy(d).to(dev)
    m = torch.empty((B,) + plan.model_shape, device=dev)
    drec = torch.empty_like(dd)
    reps = plan.deblend(dd, m, drec, batch=B, p=1.0, q=1.0, n_outer=3, n_cg=5)
    torch.cuda.synchronize()
    g = stolt.Geometry(nt, nx, DT, DX, v)
    for b in range(B):
        mo, rep = irls.irls(lambda mm: stolt.forward_irregular(g, mm, x),
                            lambda r: stolt.adjoint_irregular(g, r, x), d[b].astype(np.float64),
                            n_outer=3, n_cg=5, p=1, q=1)
        assert _rel(drec[b].cpu().numpy(), rep["d_model"]) <= 1e-3, b
        np.testing.assert_allclose(reps[b]["misfit"], rep["misfit"], rtol=1e-3)
    plan.close()


def test_irregular_at_the_benchmark_size_sampled(lib):
    """nt 1024 x nx 256 (Nt 2048, Nx 512) with 256 jittered traces and two
    velocities: the full operator pair against the oracle on one gather of a
    batch of four."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, nr, v, B = 1024, 256, 256, [1500.0, 2800.0], 4
    rng = np.random.default_rng(5)
    x = (np.arange(nr) + rng.uniform(-0.45, 0.45, nr)) * DX
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, trace_x=x, wavelet_peak_hz=25.0)
    g = stolt.Geometry(nt, nx, DT, DX, v, wavelet_peak_hz=25.0)
    m = rng.standard_normal((B,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((B, nr, nt)).astype(np.float32)
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    od, om = torch.empty_like(dd), torch.empty_like(md)
    plan.forward(md, od, batch=B)
    plan.adjoint(dd, om, batch=B)
    torch.cuda.synchronize()
    b = 2
    assert _rel(od[b].cpu().numpy(), stolt.forward_irregular(g, m[b].astype(np.float64), x)) <= 1e-4
    assert _rel(om[b].cpu().numpy(), stolt.adjoint_irregular(g, d[b].astype(np.float64), x)) <= 1e-4
    plan.close()
