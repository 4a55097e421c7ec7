"""GPU parity of the time-domain ASHRT/AASHRT pair (hyperbolic summation,
ch. 3 Table ch3_table_Radon_operators; ch. 6 Eq. ch6_AASHRT_adjoint) against
the FP64 oracle.

Tolerance.  The kernels evaluate the traveltime s = tau0/dt + sqrt(tau^2 + h^2)
(samples) in FP32: its rounding moves s by at most a few ulp of s, i.e.
< 3e-5 samples for s < 256 and < 1.2e-4 samples for s < 1024.  A shift e of
the interpolation point changes each term by e times the sample difference
of the trace, so for white-noise traces (sample differences about 1.4 times
the samples) the relative error of a sum is below about 1.5 e: 1e-4 holds for
the small cases (s < 400), 3e-4 for the full-size sample (s < 1600).
"""
import numpy as np
import pytest

from oracle import timedomain
from paper_1711_10214_gb300 import synth

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(nt, nx, v, t0, batch, seed):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt0 = 1 if t0 is None else len(t0)
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((batch, nt0, len(v), nx, nt)).astype(np.float32)
    d = rng.standard_normal((batch, nx, nt)).astype(np.float32)
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    od, om = torch.full_like(dd, np.nan), torch.full_like(md, np.nan)
    ashrt.td_forward(nt, nx, DT, DX, v, md, od, t0s=t0, batch=batch)
    ashrt.td_adjoint(nt, nx, DT, DX, v, dd, om, t0s=t0, batch=batch)
    torch.cuda.synchronize()
    return m, d, od.cpu().numpy().astype(np.float64), om.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nt,nx,v,t0,batch", [
    (64, 16, [1500.0, 2500.0], None, 1),                    # one time sample per thread
    (100, 13, [1800.0], None, 3),                           # ragged nt, nx not a multiple of the apex block
    (300, 20, [1500.0, 2300.0], [0.0, 0.05, 0.013], 2),     # two per thread, AASHRT, fractional shifts
    (700, 9, [2000.0, 3100.0], None, 1),                    # four per thread
    (1500, 5, [2500.0], [0.02], 2),                         # eight per thread
])
def test_td_pair_matches_oracle(lib, nt, nx, v, t0, batch):
    m, d, od, om = _run(nt, nx, v, t0, batch, seed=nt + nx)
    t0s = (0.0,) if t0 is None else t0
    for b in range(batch):
        ref_d = timedomain.forward(nt, nx, DT, DX, v, m[b], t0s)
        ref_m = timedomain.adjoint(nt, nx, DT, DX, v, d[b], t0s)
        assert _rel(od[b], ref_d) <= 1e-4, (b, _rel(od[b], ref_d))
        assert _rel(om[b], ref_m.reshape(om[b].shape)) <= 1e-4
    # the GPU pair is an exact transpose of itself (FP32 dot test)
    lhs = np.vdot(od, d.astype(np.float64))
    rhs = np.vdot(m.astype(np.float64), om)
    assert abs(lhs - rhs) / (np.linalg.norm(od) * np.linalg.norm(d)) <= 1e-5


def test_td_events_beyond_the_record_are_dropped(lib):
    """A large shift pushes part of every hyperbola past nt: those samples
    read and receive nothing (and nothing is written out of place)."""
    nt, nx, v, t0 = 128, 12, [1500.0], [0.4]          # tau0 = 100 samples of 128
    m, d, od, om = _run(nt, nx, v, t0, 1, seed=3)
    ref_d = timedomain.forward(nt, nx, DT, DX, v, m[0], t0)
    ref_m = timedomain.adjoint(nt, nx, DT, DX, v, d[0], t0)
    assert _rel(od[0], ref_d) <= 1e-4
    assert _rel(om[0], ref_m.reshape(om[0].shape)) <= 1e-4
    assert np.all(np.isfinite(od)) and np.all(np.isfinite(om))
    # model samples whose hyperbola starts at or past nt contribute nothing
    assert np.all(om[0, 0, 0, :, nt - 27:] == 0.0)


def test_td_full_size_sampled(lib):
    """The benchmark geometry (nt 1024, nx 256, 32 velocities, 2 gathers):
    GPU dot test over everything, and parity of the first and last velocity
    panels of gather 1 against the oracle (linearity: the other panels of the
    forward's input are zero, the oracle runs the two velocities only)."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, B = 1024, 256, 2
    v = synth.velocity_scan(1400, 3500, 32)
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev).manual_seed(11)
    m = torch.randn((B, 1, 32, nx, nt), device=dev, generator=gen)
    d = torch.randn((B, nx, nt), device=dev, generator=gen)
    od, om = torch.empty_like(d), torch.empty_like(m)
    ashrt.td_forward(nt, nx, DT, DX, v, m, od, batch=B)
    ashrt.td_adjoint(nt, nx, DT, DX, v, d, om, batch=B)
    torch.cuda.synchronize()
    lhs = torch.sum(od.double() * d.double()).item()
    rhs = torch.sum(m.double() * om.double()).item()
    assert abs(lhs - rhs) / (od.double().norm().item() * d.double().norm().item()) < 1e-5

    m1 = torch.zeros_like(m)
    m1[1, 0, 0] = m[1, 0, 0]
    m1[1, 0, 31] = m[1, 0, 31]
    ashrt.td_forward(nt, nx, DT, DX, v, m1, od, batch=B)
    torch.cuda.synchronize()
    v2 = [v[0], v[31]]
    mm = m1[1, 0][[0, 31]].cpu().numpy().astype(np.float64)
    ref_d = timedomain.forward(nt, nx, DT, DX, v2, mm[None])
    assert _rel(od[1].cpu().numpy(), ref_d) <= 3e-4
    assert float(od[0].abs().max()) == 0.0
    ref_m = timedomain.adjoint(nt, nx, DT, DX, v2, d[1].cpu().numpy().astype(np.float64))
    got = om[1, 0].cpu().numpy()[[0, 31]]
    assert _rel(got, ref_m[0]) <= 3e-4
