"""GPU blending, pseudo-deblending and sorting (ch. 2, Eqs ch2_blending and
pseudodeblending_equ) against the oracle, and the whole cube pipeline:
shots -> blended records -> pseudo-deblended shots -> receiver gathers ->
robust IRLS deblend -> shot gathers.

Bars: the copies (pseudo-deblending of a given record, sorting) bit-exact;
blending (FP32 sums of a few shots in shot order) to 1e-6 relative; the
pipeline's Q within 0.1 dB of the oracle pipeline's (the IRLS bar)."""
import numpy as np
import pytest

from oracle import blending, irls, stolt
from paper_1711_10214_gb300 import synth

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_blend_pseudo_deblend_sort_match_oracle(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(0)
    ns, nr, nt, nb = 13, 5, 50, 300
    D = rng.standard_normal((ns, nr, nt)).astype(np.float32)
    fire = np.array([-7, 0, 20, 21, 60, 95, 95, 130, 170, 200, 230, 262, 290], np.int32)
    Dd, fd = torch.from_numpy(D).to(dev), torch.from_numpy(fire).to(dev)
    b = torch.full((nr, nb), np.nan, device=dev)
    ashrt.blend(Dd, fd, b)
    Dt = torch.full_like(Dd, np.nan)
    ashrt.pseudo_deblend(b, fd, Dt)
    S = torch.full((nr, ns, nt), np.nan, device=dev)
    ashrt.sort_gathers(Dt, S)
    torch.cuda.synchronize()
    bh = b.cpu().numpy()
    assert _rel(bh, blending.blend(D, fire, nb)) <= 1e-6
    Dth = Dt.cpu().numpy()
    assert np.array_equal(Dth, blending.pseudo_deblend(bh, fire, nt).astype(np.float32))
    assert np.array_equal(S.cpu().numpy(), blending.sort_gathers(Dth))
    # the GPU pair is a transpose pair (dot test in FP64 of the FP32 results)
    r = rng.standard_normal((nr, nb)).astype(np.float32)
    ashrt.pseudo_deblend(torch.from_numpy(r).to(dev), fd, Dt)
    torch.cuda.synchronize()
    lhs = np.vdot(bh.astype(np.float64), r.astype(np.float64))
    rhs = np.vdot(D.astype(np.float64), Dt.cpu().numpy().astype(np.float64))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(bh) * np.linalg.norm(r)


def test_sort_rejects_in_place(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    x = torch.zeros((3, 3, 8), device=torch.device("cuda:0"))
    with pytest.raises(ashrt.AshrtError):
        ashrt.sort_gathers(x, x)


def _cube(ns, nr, nt, seed):
    """Common-shot gathers of three flat reflectors: the traveltime
    sqrt(tau^2 + ((x_s - x_r)/v)^2) is a hyperbola with its apex at the
    receiver in every receiver gather."""
    xs = np.arange(ns) * DX
    xr = (np.arange(nr) * 8 + 4) * DX
    t = np.arange(nt) * DT
    D = np.zeros((ns, nr, nt))
    for i in range(ns):
        for j in range(nr):
            for tau, v, A in ((0.10, 1600.0, 1.0), (0.22, 2000.0, -0.7), (0.34, 2400.0, 0.6)):
                D[i, j] += A * synth.ricker(t - np.sqrt(tau * tau + ((xs[i] - xr[j]) / v) ** 2),
                                            25.0)
    rng = np.random.default_rng(seed)
    fire = (np.arange(ns) * (nt // 2) + rng.integers(0, nt // 4, ns)).astype(np.int32)
    return D, fire


def test_cube_pipeline_matches_oracle_and_deblends(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    ns, nr, nt = 32, 2, 128
    D, fire = _cube(ns, nr, nt, seed=7)
    nb = int(fire.max()) + nt
    v = synth.velocity_scan(1400, 3000, 8)
    dev = torch.device("cuda:0")
    Dd, fd = torch.from_numpy(D.astype(np.float32)).to(dev), torch.from_numpy(fire).to(dev)
    b = torch.empty((nr, nb), device=dev)
    Dt = torch.empty_like(Dd)
    crg = torch.empty((nr, ns, nt), device=dev)
    ashrt.blend(Dd, fd, b)
    ashrt.pseudo_deblend(b, fd, Dt)
    ashrt.sort_gathers(Dt, crg)
    plan = ashrt.Plan(nt, ns, DT, DX, v, wavelet_peak_hz=25.0, max_batch=nr, with_solver=True)
    m = torch.empty((nr,) + plan.model_shape, device=dev)
    rec_crg = torch.empty_like(crg)
    plan.deblend(crg, m, rec_crg, batch=nr, p=1.0, q=1.0, n_outer=5, n_cg=20)
    rec = torch.empty_like(Dd)
    ashrt.sort_gathers(rec_crg, rec)
    torch.cuda.synchronize()
    plan.close()

    crg_h, rec_h = crg.cpu().numpy().astype(np.float64), rec.cpu().numpy().astype(np.float64)
    clean_crg = blending.sort_gathers(D)
    pd_ref = blending.sort_gathers(blending.pseudo_deblend(blending.blend(D, fire, nb), fire, nt))
    assert _rel(crg_h, pd_ref) <= 1e-6
    g = stolt.Geometry(nt, ns, DT, DX, v, wavelet_peak_hz=25.0)
    rec_crg_h = blending.sort_gathers(rec_h)
    for j in range(nr):
        _, rep = irls.irls(lambda mm: stolt.forward(g, mm), lambda dd: stolt.adjoint(g, dd),
                           pd_ref[j], 5, 20)
        q_pd = irls.q_db(clean_crg[j], pd_ref[j])
        q_ref = irls.q_db(clean_crg[j], rep["d_model"])
        q_gpu = irls.q_db(clean_crg[j], rec_crg_h[j])
        assert abs(q_gpu - q_ref) <= 0.1, (j, q_gpu, q_ref)
        assert q_gpu - q_pd > 2.0, (j, q_gpu, q_pd)
