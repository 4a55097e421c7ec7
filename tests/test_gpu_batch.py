"""Uneven batches (gathers of different trace counts in one call) and the
recorded-graph solve, against the FP64 oracle gather by gather."""
import numpy as np
import pytest

from oracle import irls, stolt

pytestmark = pytest.mark.gpu
DT, DX = 0.004, 12.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _packed(rng, nxs, nt, P):
    ms = [rng.standard_normal((P, nx, nt)) for nx in nxs]
    ds = [rng.standard_normal((nx, nt)) for nx in nxs]
    return ms, ds, np.concatenate([m.ravel() for m in ms]), np.concatenate([d.ravel() for d in ds])


def _split(flat, shapes):
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(flat[o:o + n].reshape(s))
        o += n
    return out


@pytest.mark.parametrize("max_resident", [64, 2])
def test_uneven_operator_parity(lib, max_resident):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nxs, v, t0 = 64, [13, 20, 9, 31, 17], [1600.0, 2500.0], [0.0, 0.03]
    P = len(v) * len(t0)
    b = ashrt.Batch(nt, nxs, DT, DX, v, t0s=t0, max_resident=max_resident)
    assert b.n_classes == 2
    rng = np.random.default_rng(21)
    ms, ds, mflat, dflat = _packed(rng, nxs, nt, P)
    dev = torch.device("cuda:0")
    mg = torch.from_numpy(mflat.astype(np.float32)).to(dev)
    dg = torch.from_numpy(dflat.astype(np.float32)).to(dev)
    od, om = torch.empty_like(dg), torch.empty_like(mg)
    b.forward(mg, od)
    b.adjoint(dg, om)
    torch.cuda.synchronize()
    od_l = _split(od.cpu().numpy().astype(np.float64), [(nx, nt) for nx in nxs])
    om_l = _split(om.cpu().numpy().astype(np.float64), [(P, nx, nt) for nx in nxs])
    for i, nx in enumerate(nxs):
        g = stolt.Geometry(nt, nx, DT, DX, v, t0s=t0)
        m32 = ms[i].astype(np.float32).astype(np.float64).reshape(g.model_shape)
        d32 = ds[i].astype(np.float32).astype(np.float64)
        assert _rel(od_l[i], stolt.forward(g, m32)) <= 1e-4, i
        assert _rel(om_l[i].reshape(g.model_shape), stolt.adjoint(g, d32)) <= 1e-4, i
    b.close()


def test_uneven_deblend_matches_oracle(lib):
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nxs, v = 72, [11, 24, 19], [1500.0, 2400.0]
    b = ashrt.Batch(nt, nxs, DT, DX, v, with_solver=True, max_resident=2)
    rng = np.random.default_rng(22)
    ds = [rng.standard_normal((nx, nt)) for nx in nxs]
    dflat = np.concatenate([d.ravel() for d in ds]).astype(np.float32)
    dev = torch.device("cuda:0")
    dg = torch.from_numpy(dflat).to(dev)
    mg = torch.empty(b.model_elems, device=dev)
    rg = torch.empty_like(dg)
    reps = b.deblend(dg, mg, rg, p=1.0, q=1.0, n_outer=3, n_cg=5)
    torch.cuda.synchronize()
    rec = _split(rg.cpu().numpy().astype(np.float64), [(nx, nt) for nx in nxs])
    for i, nx in enumerate(nxs):
        g = stolt.Geometry(nt, nx, DT, DX, v)
        d64 = ds[i].astype(np.float32).astype(np.float64)
        m, rep = irls.irls(lambda x: stolt.forward(g, x), lambda r: stolt.adjoint(g, r), d64,
                           n_outer=3, n_cg=5, p=1, q=1)
        assert _rel(rec[i], stolt.forward(g, m)) <= 1e-3, i
        np.testing.assert_allclose(reps[i]["misfit"], rep["misfit"], rtol=1e-3)
    b.close()


def test_recorded_graph_solve_matches_direct(lib):
    """use_graph records the whole IRLS/CGLS sequence once and replays it;
    results equal the directly launched solve (up to the order of FP64
    atomic additions in the norms)."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nt, nx, v, B = 96, 24, [1500.0, 2300.0, 3100.0], 3
    plan = ashrt.Plan(nt, nx, DT, DX, v, max_batch=B, with_solver=True)
    rng = np.random.default_rng(23)
    dev = torch.device("cuda:0")
    d = torch.from_numpy(rng.standard_normal((B, nx, nt)).astype(np.float32)).to(dev)
    m0, m1 = torch.empty((B,) + plan.model_shape, device=dev), torch.empty((B,) + plan.model_shape, device=dev)
    r0, r1 = torch.empty_like(d), torch.empty_like(d)
    kw = dict(p=1.0, q=1.0, n_outer=3, n_cg=6)
    rep0 = plan.deblend(d, m0, r0, batch=B, **kw)
    n_before = ashrt.kernel_launches()
    rep1 = plan.deblend(d, m1, r1, batch=B, use_graph=1, **kw)      # records and replays
    rep2 = plan.deblend(d, m1, r1, batch=B, use_graph=1, **kw)      # replays
    torch.cuda.synchronize()
    assert ashrt.kernel_launches() > n_before
    assert _rel(r1.cpu().numpy(), r0.cpu().numpy()) < 1e-5
    assert _rel(m1.cpu().numpy(), m0.cpu().numpy()) < 1e-4
    for a, c in zip(rep0, rep2):
        assert a["applies_fwd"] == c["applies_fwd"] and a["outer_done"] == c["outer_done"]
        np.testing.assert_allclose(a["misfit"], c["misfit"], rtol=1e-5)
    plan.close()


def test_uneven_sample_counts(lib):
    """Gathers of different nt and nx in one batch: classes per (nt, Nx);
    operator parity and the deblend of every gather as if alone."""
    import torch
    from paper_1711_10214_gb300 import ashrt
    nts, nxs, v = [64, 80, 64, 72, 80], [13, 20, 9, 17, 11], [1600.0, 2500.0]
    b = ashrt.Batch(nts, nxs, DT, DX, v, with_solver=True, max_resident=2)
    assert b.n_classes == 4     # (nt, Nx): (64, 32) twice, (80, 64), (72, 64), (80, 32)
    rng = np.random.default_rng(24)
    ms = [rng.standard_normal((2, nx, nt)) for nt, nx in zip(nts, nxs)]
    ds = [rng.standard_normal((nx, nt)) for nt, nx in zip(nts, nxs)]
    mflat = np.concatenate([m.ravel() for m in ms]).astype(np.float32)
    dflat = np.concatenate([d.ravel() for d in ds]).astype(np.float32)
    assert (b.model_elems, b.data_elems) == (mflat.size, dflat.size)
    dev = torch.device("cuda:0")
    mg, dg = torch.from_numpy(mflat).to(dev), torch.from_numpy(dflat).to(dev)
    od, om = torch.empty_like(dg), torch.empty_like(mg)
    b.forward(mg, od)
    b.adjoint(dg, om)
    mrec, drec = torch.empty_like(mg), torch.empty_like(dg)
    reps = b.deblend(dg, mrec, drec, p=1.0, q=1.0, n_outer=2, n_cg=4)
    torch.cuda.synchronize()
    od_l = _split(od.cpu().numpy().astype(np.float64), [(nx, nt) for nt, nx in zip(nts, nxs)])
    om_l = _split(om.cpu().numpy().astype(np.float64), [(2, nx, nt) for nt, nx in zip(nts, nxs)])
    rec = _split(drec.cpu().numpy().astype(np.float64), [(nx, nt) for nt, nx in zip(nts, nxs)])
    for i, (nt, nx) in enumerate(zip(nts, nxs)):
        g = stolt.Geometry(nt, nx, DT, DX, v)
        m32 = ms[i].astype(np.float32).astype(np.float64).reshape(g.model_shape)
        d32 = ds[i].astype(np.float32).astype(np.float64)
        assert _rel(od_l[i], stolt.forward(g, m32)) <= 1e-4, i
        assert _rel(om_l[i].reshape(g.model_shape), stolt.adjoint(g, d32)) <= 1e-4, i
        mo, rep = irls.irls(lambda x: stolt.forward(g, x), lambda r: stolt.adjoint(g, r), d32,
                            n_outer=2, n_cg=4, p=1, q=1)
        assert _rel(rec[i], stolt.forward(g, mo)) <= 1e-3, i
        np.testing.assert_allclose(reps[i]["misfit"], rep["misfit"], rtol=1e-3)
    b.close()


def test_c4_gathers_through_the_batch_layer(lib):
    """Gathers of the uneven workload's own generator (nt 1500 at 4 ms, 5-40
    events, three dithered interfering sources, 25 Hz wavelet), narrowed to
    small trace counts and two scan velocities so that the FP64 oracle
    finishes in seconds, deblended through the batch layer as the workload
    runs it: classes per padded width (Nx 64 and 128 here, Nt 4096: the
    radix-16 forward rows), every class's kernels autotuned, one gather
    resident at a time so each class streams in chunks, and the recorded
    graph replayed from chunk to chunk on new data.  Each gather must match
    the oracle IRLS of that gather alone (ch. 1: gathers are independent)."""
    import torch
    from paper_1711_10214_gb300 import ashrt, synth
    nt, nxs, v = 1500, [20, 37, 26, 48], [1600.0, 2600.0]
    c = synth.config4(range(4), nxs, nt=nt)
    b = ashrt.Batch(nt, nxs, DT, DX, v, wavelet_peak_hz=c["f_peak"], max_resident=1,
                    with_solver=True)
    assert b.n_classes == 2
    b.autotune()
    dev = torch.device("cuda:0")
    dg = torch.from_numpy(c["blended"]).to(dev)
    mg = torch.empty(b.model_elems, device=dev)
    rg = torch.empty_like(dg)
    kw = dict(p=1.0, q=1.0, n_outer=2, n_cg=4)
    b.deblend(dg, mg, rg, use_graph=1, **kw)
    rg.fill_(float("nan"))
    reps = b.deblend(dg, mg, rg, use_graph=1, **kw)         # replays the recorded graphs
    torch.cuda.synchronize()
    rec = _split(rg.cpu().numpy().astype(np.float64), [(nx, nt) for nx in nxs])
    ds = _split(c["blended"].astype(np.float64), [(nx, nt) for nx in nxs])
    for i, nx in enumerate(nxs):
        g = stolt.Geometry(nt, nx, DT, DX, v, wavelet_peak_hz=c["f_peak"])
        assert (g.Nt, g.Nx) == (4096, 64 if nx <= 32 else 128)
        m, rep = irls.irls(lambda x: stolt.forward(g, x), lambda r: stolt.adjoint(g, r), ds[i],
                           **kw)
        assert _rel(rec[i], rep["d_model"]) <= 1e-3, (i, _rel(rec[i], rep["d_model"]))
        np.testing.assert_allclose(reps[i]["misfit"], rep["misfit"], rtol=1e-3)
    b.close()
