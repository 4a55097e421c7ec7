"""Edge and degenerate cases of the operator pair and the robust solve.

* the smallest gathers (nt 2..5, nx 2..3), where the plan's minimum padded
  sizes (Nt >= 64, Nx >= 16) exceed twice the gather: parity with the FP64
  oracle on the same padded grid, and the dot test;
* zero models and zero data map to exact zeros;
* an all-zero gather in the robust solve (MAD = 0, max|m| = 0: the eps
  fall-backs) returns zeros with finite misfits and no error, beside a
  normal gather in the same batch;
* batch sizes outside [1, max_batch] are rejected.
"""
import numpy as np
import pytest

from oracle import irls, stolt

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nt,nx", [(2, 2), (5, 3), (3, 2)])
def test_smallest_gathers_match_the_oracle(lib, nt, nx):
    import torch
    from paper_1711_10214_gb300 import ashrt
    v = [1500.0, 2600.0]
    plan = ashrt.Plan(nt, nx, DT, DX, v)
    assert (plan.Nt, plan.Nx) == (64, 16)      # the minimum padded sizes
    g = stolt.Geometry(nt, nx, DT, DX, v, Nt=plan.Nt, Nx=plan.Nx)
    rng = np.random.default_rng(nt * 10 + nx)
    m = rng.standard_normal((1,) + g.model_shape).astype(np.float32)
    d = rng.standard_normal((1,) + g.data_shape).astype(np.float32)
    dev = torch.device("cuda:0")
    md, dd = torch.from_numpy(m).to(dev), torch.from_numpy(d).to(dev)
    od, om = torch.empty_like(dd), torch.empty_like(md)
    plan.forward(md, od)
    plan.adjoint(dd, om)
    torch.cuda.synchronize()
    od, om = od.cpu().numpy().astype(np.float64), om.cpu().numpy().astype(np.float64)
    assert _rel(od[0], stolt.forward(g, m[0].astype(np.float64))) <= 1e-4
    assert _rel(om[0], stolt.adjoint(g, d[0].astype(np.float64))) <= 1e-4
    dot = abs(np.vdot(od, d) - np.vdot(m, om)) / (np.linalg.norm(od) * np.linalg.norm(d))
    assert dot <= 1e-5
    plan.close()


def test_zero_inputs_map_to_exact_zeros(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, B = 96, 24, 2
    plan = ashrt.Plan(nt, nx, DT, DX, [1500.0, 2500.0], t0s=[0.0, 0.05], max_batch=B,
                      wavelet_peak_hz=25.0)
    dev = torch.device("cuda:0")
    m = torch.zeros((B,) + plan.model_shape, device=dev)
    d = torch.zeros((B, nx, nt), device=dev)
    od = torch.full_like(d, 7.0)
    om = torch.full_like(m, 7.0)
    plan.forward(m, od, batch=B)
    plan.adjoint(d, om, batch=B)
    torch.cuda.synchronize()
    assert float(od.abs().max()) == 0.0 and float(om.abs().max()) == 0.0
    plan.close()


def test_all_zero_gather_in_the_robust_solve(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, B = 80, 20, [1600.0, 2500.0], 2
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, with_solver=True)
    g = stolt.Geometry(nt, nx, DT, DX, v)
    rng = np.random.default_rng(17)
    d = np.zeros((B, nx, nt))
    d[1] = rng.standard_normal((nx, nt))
    dev = torch.device("cuda:0")
    dd = torch.from_numpy(d.astype(np.float32)).to(dev)
    m = torch.full((B,) + plan.model_shape, 3.0, device=dev)
    drec = torch.full_like(dd, 3.0)
    reps = plan.deblend(dd, m, drec, batch=B, p=1.0, q=1.0, n_outer=3, n_cg=6)
    torch.cuda.synchronize()
    assert float(m[0].abs().max()) == 0.0 and float(drec[0].abs().max()) == 0.0
    assert all(np.isfinite(reps[0]["misfit"])) and reps[0]["misfit"][-1] == 0.0
    # the other gather of the batch is solved as if alone
    mo, _ = irls.irls(lambda x: stolt.forward(g, x), lambda r: stolt.adjoint(g, r),
                      d[1].astype(np.float32).astype(np.float64), n_outer=3, n_cg=6, p=1, q=1)
    assert _rel(drec[1].cpu().numpy().astype(np.float64), stolt.forward(g, mo)) <= 1e-3
    plan.close()


def test_batch_outside_the_plan_is_rejected(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    plan = ashrt.Plan(64, 16, DT, DX, [2000.0], max_batch=2)
    dev = torch.device("cuda:0")
    m = torch.zeros((3,) + plan.model_shape, device=dev)
    d = torch.zeros((3, 16, 64), device=dev)
    for b in (0, 3):
        with pytest.raises(ashrt.AshrtError) as e:
            plan.forward(m, d, batch=b)
        assert e.value.status == 1
        with pytest.raises(ashrt.AshrtError):
            plan.adjoint(d, m, batch=b)
    plan.close()
