"""GPU robust IRLS deblending against the FP64 oracle IRLS (ch. 4).

Separated (recovered) gathers within relative l2 1e-3 of the oracle's and Q
within 0.1 dB, on config 1 (nt 256, nx 64, 8 velocities, 5 x 20, p = q = 1)
and on smaller ragged cases covering p/q variants, mu > 0, trace masks with
dead traces (median over live samples only), the stopping rule and batches.
"""
import numpy as np
import pytest

from oracle import irls, stolt
from paper_1711_10214_gb300 import synth

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5
SEP_TOL = 1e-3


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(torch, plan, d, mask=None, **kw):
    dev = torch.device("cuda:0")
    B = d.shape[0]
    dd = torch.from_numpy(d.astype(np.float32)).to(dev)
    m = torch.empty((B,) + plan.model_shape, device=dev)
    drec = torch.empty_like(dd)
    mk = None if mask is None else torch.from_numpy(mask.astype(np.float32)).to(dev)
    reps = plan.deblend(dd, m, drec, batch=B, mask=mk, **kw)
    torch.cuda.synchronize()
    return m.cpu().numpy().astype(np.float64), drec.cpu().numpy().astype(np.float64), reps


def _oracle(g, d, mask=None, **kw):
    if mask is None:
        f = lambda m: stolt.forward(g, m)
        t = lambda r: stolt.adjoint(g, r)
        live = None
    else:
        f = lambda m: stolt.forward(g, m, mask)
        t = lambda r: stolt.adjoint(g, r, mask)
        live = np.broadcast_to(mask[:, None] != 0, d.shape)
    m, rep = irls.irls(f, t, d, live=live, **kw)
    return m, stolt.forward(g, m), rep


def test_config1_deblend_parity(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    c = synth.config1(0)
    plan = ashrt.Plan(c["nt"], c["nx"], DT, DX, c["velocities"], wavelet_peak_hz=c["f_peak"],
                      with_solver=True)
    g = stolt.Geometry(c["nt"], c["nx"], DT, DX, c["velocities"], wavelet_peak_hz=c["f_peak"])
    d = c["blended"][None].astype(np.float32)
    _, drec, reps = _run(torch, plan, d, p=1.0, q=1.0, n_outer=5, n_cg=20)
    _, drec_o, rep_o = _oracle(g, d[0].astype(np.float64), n_outer=5, n_cg=20, p=1, q=1)
    assert _rel(drec[0], drec_o) <= SEP_TOL, _rel(drec[0], drec_o)
    q_gpu = irls.q_db(c["clean"], drec[0])
    q_or = irls.q_db(c["clean"], drec_o)
    assert abs(q_gpu - q_or) <= 0.1, (q_gpu, q_or)
    np.testing.assert_allclose(reps[0]["misfit"], rep_o["misfit"], rtol=1e-3)
    plan.close()


@pytest.mark.parametrize("kw", [
    dict(p=2.0, q=2.0, n_outer=1, n_cg=8),
    dict(p=1.0, q=2.0, n_outer=3, n_cg=6),
    dict(p=2.0, q=1.0, n_outer=3, n_cg=6, b_m=2.0),
    dict(p=1.0, q=1.0, n_outer=3, n_cg=6, mu=0.05),
    dict(p=1.0, q=1.0, n_outer=3, n_cg=6, warm_start_cg=0),
    dict(p=1.5, q=1.2, n_outer=3, n_cg=5),
])
def test_small_variants(lib, kw):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v = 90, 21, [1500.0, 2400.0]
    rng = np.random.default_rng(11)
    B = 2
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, with_solver=True)
    g = stolt.Geometry(nt, nx, DT, DX, v)
    d = rng.standard_normal((B, nx, nt))
    d[:, :, :10] = 0.0          # exact zeros: ties in the median
    _, drec, reps = _run(torch, plan, d, **kw)
    okw = {k: v for k, v in kw.items() if k != "warm_start_cg"}
    okw["warm_start"] = bool(kw.get("warm_start_cg", 1))
    for b in range(B):
        _, drec_o, rep_o = _oracle(g, d[b], **okw)
        assert _rel(drec[b], drec_o) <= SEP_TOL, (b, _rel(drec[b], drec_o))


def test_masked_interpolation_and_dead_traces(lib):
    """Sampling operator S (ch. 6): dead traces are excluded from the
    residual median/MAD and from the misfit."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, t0 = 80, 24, [1800.0, 2600.0], [0.0, 0.04]
    rng = np.random.default_rng(12)
    plan = ashrt.Plan(nt, nx, DT, DX, v, t0s=t0, with_solver=True)
    g = stolt.Geometry(nt, nx, DT, DX, v, t0s=t0)
    mask = (rng.random(nx) < 0.5).astype(np.float64)
    d = rng.standard_normal((1, nx, nt)) * mask[None, :, None]
    _, drec, reps = _run(torch, plan, d, mask=mask[None], p=1.0, q=1.0, n_outer=3, n_cg=6)
    _, drec_o, rep_o = _oracle(g, d[0], mask=mask, n_outer=3, n_cg=6, p=1, q=1)
    assert _rel(drec[0], drec_o) <= SEP_TOL
    np.testing.assert_allclose(reps[0]["misfit"], rep_o["misfit"], rtol=1e-3)


def test_stopping_rule(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v = 64, 16, [2000.0]
    rng = np.random.default_rng(13)
    plan = ashrt.Plan(nt, nx, DT, DX, v, with_solver=True)
    g = stolt.Geometry(nt, nx, DT, DX, v)
    d = rng.standard_normal((1, nx, nt))
    _, _, reps = _run(torch, plan, d, p=1.0, q=2.0, n_outer=20, n_cg=4, tol=0.05)
    _, _, rep_o = _oracle(g, d[0], n_outer=20, n_cg=4, p=1, q=2, tol=0.05)
    assert reps[0]["outer_done"] == rep_o["outer_done"] < 20
    assert reps[0]["flags"] & 1


def test_nonfinite_input_is_rejected(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    plan = ashrt.Plan(64, 16, DT, DX, [2000.0], with_solver=True)
    d = torch.zeros((1, 16, 64), device="cuda:0")
    d[0, 3, 7] = float("nan")
    m = torch.empty((1, 1, 1, 16, 64), device="cuda:0")
    with pytest.raises(ashrt.AshrtError) as e:
        plan.deblend(d, m)
    assert e.value.status == 4


@pytest.mark.parametrize("use_m0,use_wr0", [(True, False), (False, True), (True, True)])
def test_warm_start_parity(lib, use_m0, use_wr0):
    """Warm start from a given model m0 and/or residual weights W_r0 (the
    inputs a learned predictor supplies) against the oracle's warm start."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, B = 80, 20, [1600.0, 2500.0], 2
    rng = np.random.default_rng(14)
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, with_solver=True)
    g = stolt.Geometry(nt, nx, DT, DX, v)
    d = rng.standard_normal((B, nx, nt))
    m0 = 0.1 * rng.standard_normal((B,) + g.model_shape)
    wr0 = rng.uniform(0.3, 1.5, (B, nx, nt))
    dev = torch.device("cuda:0")
    m0g = torch.from_numpy(m0.astype(np.float32)).to(dev) if use_m0 else None
    wr0g = torch.from_numpy(wr0.astype(np.float32)).to(dev) if use_wr0 else None
    _, drec, reps = _run(torch, plan, d, p=1.0, q=1.0, n_outer=3, n_cg=6, m0=m0g, wr0=wr0g)
    for b in range(B):
        f = lambda m: stolt.forward(g, m)
        t = lambda r: stolt.adjoint(g, r)
        m, rep = irls.irls(f, t, d[b].astype(np.float32).astype(np.float64), n_outer=3, n_cg=6,
                           p=1, q=1,
                           m0=m0[b].astype(np.float32).astype(np.float64) if use_m0 else None,
                           wr0=wr0[b].astype(np.float32).astype(np.float64) if use_wr0 else None)
        assert _rel(drec[b], stolt.forward(g, m)) <= SEP_TOL, b
        np.testing.assert_allclose(reps[b]["misfit"], rep["misfit"], rtol=1e-3)
    plan.close()


def test_unpadded_grid_deblend_parity(lib):
    """pad_t = pad_x = 1 (nt 92 -> Nt 128, nx 21 -> Nx 32): the model and the
    data fill more than half of each transform, so the kernels run their
    general forms (the row kernels' full first pass, the trace-axis c2r with
    its weight tile forming every output of its last pass, the TMA-fed r2c
    with its fused CG update reading every row; nt is a multiple of 4 so that
    both staged forms apply); the solve against the oracle IRLS."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, B = 92, 21, [1500.0, 2400.0], 2
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, with_solver=True, pad_t=1, pad_x=1)
    g = stolt.Geometry(nt, nx, DT, DX, v, pad_t=1, pad_x=1)
    assert (plan.Nt, plan.Nx) == (g.Nt, g.Nx) == (128, 32)
    rng = np.random.default_rng(12)
    d = rng.standard_normal((B, nx, nt))
    _, drec, _ = _run(torch, plan, d, p=1.0, q=1.0, n_outer=3, n_cg=6)
    for b in range(B):
        _, drec_o, _ = _oracle(g, d[b], p=1.0, q=1.0, n_outer=3, n_cg=6)
        assert _rel(drec[b], drec_o) <= SEP_TOL, (b, _rel(drec[b], drec_o))
