"""ashrt_forward_static, the allocation-free forward operator.

It serves callers that cannot allocate device memory (a host application
that owns the GPU's memory and passes only its input/output buffers, or a
latency-critical loop where cudaMalloc would synchronise the device).  The
test calls it through the C ABI twice in a row, on different inputs and
shapes, and checks each result against ashrt_forward (the plan-based entry
point) within the operator tolerance of the other tests; it also checks that
a call too large for the static scratch is refused with a clear error.  It
lives in its own file, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5
TOL = 1e-4


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forward_static_matches_plan_forward():
    import torch
    from paper_1711_10214_gb300 import ashrt
    ashrt.load()
    dev = torch.device("cuda:0")
    cases = [
        dict(nt=256, nx=64, v=[1500.0, 1900.0, 2500.0, 3000.0], t0=None, batch=2,
             kw=dict(wavelet_peak_hz=20.0)),
        dict(nt=120, nx=30, v=[1700.0, 2600.0], t0=[0.0, 0.05], batch=3, kw={}),
    ]
    for i, c in enumerate(cases):     # two calls in a row through the shared static scratch
        rng = np.random.default_rng(40 + i)
        nt0 = 1 if c["t0"] is None else len(c["t0"])
        m = torch.from_numpy(rng.standard_normal(
            (c["batch"], nt0, len(c["v"]), c["nx"], c["nt"])).astype(np.float32)).to(dev)
        mask = torch.from_numpy((rng.random((c["batch"], c["nx"])) < 0.7).astype(np.float32)).to(dev)
        plan = ashrt.Plan(c["nt"], c["nx"], DT, DX, c["v"], t0s=c["t0"], max_batch=c["batch"],
                          **c["kw"])
        ref = torch.empty((c["batch"], c["nx"], c["nt"]), device=dev)
        plan.forward(m, ref, mask=mask, batch=c["batch"])
        out = torch.full_like(ref, float("nan"))
        ashrt.forward_static(c["nt"], c["nx"], DT, DX, c["v"], m, out, t0s=c["t0"], mask=mask,
                             batch=c["batch"], **c["kw"])
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= TOL
        plan.close()


def test_forward_static_rejects_oversize():
    import torch
    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda:0")
    m = torch.zeros((1, 1, 8, 256, 1024), device=dev)
    d = torch.zeros((1, 256, 1024), device=dev)
    with pytest.raises(ashrt.AshrtError) as e:
        ashrt.forward_static(1024, 256, DT, DX, [1500.0] * 8, m, d)
    assert e.value.status == 1 and "static scratch" in str(e.value)
