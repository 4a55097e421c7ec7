"""ashrt_forward_static, the allocation-free forward operator.

It serves callers that cannot allocate device memory (a host application
that owns the GPU's memory and passes only its input/output buffers, or a
latency-critical loop where cudaMalloc would synchronise the device).  The
test calls it through the C ABI several times in a row on different inputs
and shapes, sharing the one static scratch array: a large call first, then a
smaller one whose nt is not a multiple of 4 (so the padding columns of the
spectrum rows hold what the previous call left there).  Each result is
checked against the FP64 oracle and against ashrt_forward (the plan-based
entry point) within the operator tolerance of the other tests.  Repeating the
calls leaves the device's free memory unchanged (the first round has loaded
every kernel).  A call too large for the scratch and a call made while the
stream is being captured into a CUDA graph are refused with clear errors.
It lives in its own file, collected last.
"""
import numpy as np
import pytest

from oracle import stolt

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5
TOL = 1e-4

CASES = [
    dict(nt=256, nx=64, v=[1500.0, 1900.0, 2500.0, 3000.0], t0=None, batch=2,
         kw=dict(wavelet_peak_hz=20.0)),
    dict(nt=125, nx=30, v=[1700.0, 2600.0], t0=[0.0, 0.05], batch=3, kw={}),
    dict(nt=120, nx=30, v=[1700.0, 2600.0], t0=[0.0, 0.05], batch=3, kw=dict(fmax_hz=60.0)),
]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inputs(torch, c, seed):
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(seed)
    nt0 = 1 if c["t0"] is None else len(c["t0"])
    m = rng.standard_normal((c["batch"], nt0, len(c["v"]), c["nx"], c["nt"])).astype(np.float32)
    mask = (rng.random((c["batch"], c["nx"])) < 0.7).astype(np.float32)
    return m, mask, torch.from_numpy(m).to(dev), torch.from_numpy(mask).to(dev)


def test_forward_static_matches_oracle_and_plan(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda:0")
    bufs = []
    for i, c in enumerate(CASES):
        m, mask, md, maskd = _inputs(torch, c, 40 + i)
        out = torch.full((c["batch"], c["nx"], c["nt"]), float("nan"), device=dev)
        bufs.append((c, m, mask, md, maskd, out))
    refs = []
    for c, m, mask, md, maskd, out in bufs:          # calls in a row through the shared scratch
        ashrt.forward_static(c["nt"], c["nx"], DT, DX, c["v"], md, out, t0s=c["t0"],
                             mask=maskd, batch=c["batch"], **c["kw"])
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        g = stolt.Geometry(c["nt"], c["nx"], DT, DX, c["v"],
                           t0s=(0.0,) if c["t0"] is None else c["t0"], **c["kw"])
        ref = stolt.forward_batch(g, m.astype(np.float64), mask.astype(np.float64))
        assert _rel(got, ref) <= TOL, (c["nt"], _rel(got, ref))
        plan = ashrt.Plan(c["nt"], c["nx"], DT, DX, c["v"], t0s=c["t0"], max_batch=c["batch"],
                          **c["kw"])
        pd = torch.empty_like(out)
        plan.forward(md, pd, mask=maskd, batch=c["batch"])
        torch.cuda.synchronize()
        assert _rel(got, pd.cpu().numpy().astype(np.float64)) <= TOL
        plan.close()
        refs.append(got)
    # the same calls again: no device memory is taken, and the results repeat
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for (c, m, mask, md, maskd, out), got in zip(bufs, refs):
        out.fill_(float("nan"))
        ashrt.forward_static(c["nt"], c["nx"], DT, DX, c["v"], md, out, t0s=c["t0"],
                             mask=maskd, batch=c["batch"], **c["kw"])
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy().astype(np.float64), got) <= 1e-6
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_forward_static_rejects_oversize(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda:0")
    m = torch.zeros((1, 1, 8, 256, 1024), device=dev)
    d = torch.zeros((1, 256, 1024), device=dev)
    with pytest.raises(ashrt.AshrtError) as e:
        ashrt.forward_static(1024, 256, DT, DX, [1500.0] * 8, m, d)
    assert e.value.status == 1 and "static scratch" in str(e.value)


def test_forward_static_refuses_stream_capture(lib):
    """Its tables are uploaded from host memory that lives only for the call,
    which a captured graph would read at replay: the call is refused while its
    stream is capturing, and works again afterwards."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda:0")
    c = CASES[1]
    m, mask, md, maskd = _inputs(torch, c, 7)
    out = torch.zeros((c["batch"], c["nx"], c["nt"]), device=dev)
    s = torch.cuda.Stream(dev)
    graph = torch.cuda.CUDAGraph()
    err = None
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s):
        try:
            ashrt.forward_static(c["nt"], c["nx"], DT, DX, c["v"], md, out, t0s=c["t0"],
                                 mask=maskd, batch=c["batch"], stream=s)
        except ashrt.AshrtError as e:
            err = e
        out.add_(0.0)                 # the captured graph is not empty
    assert err is not None and err.status == 1 and "capture" in str(err)
    ashrt.forward_static(c["nt"], c["nx"], DT, DX, c["v"], md, out, t0s=c["t0"], mask=maskd,
                         batch=c["batch"])
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
