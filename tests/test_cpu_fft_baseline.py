"""The scipy.fft CPU baseline of the measurement computes the same operator
as the FP64 oracle (so that its timing is a fair comparison): forward and
adjoint on small gathers with the wavelet and asymptote shifts, in FP64
(1e-10) and FP32 (1e-4), and its pair is an exact transpose."""
import numpy as np
import pytest

import bench
from oracle import stolt

DT, DX = 0.004, 12.5


@pytest.mark.parametrize("nt,nx,v,t0,fp", [
    (64, 16, [1500.0, 2600.0], (0.0,), 0.0),
    (50, 13, [1800.0], (0.0, 0.03), 25.0),
    (96, 24, [0.0, 1700.0, 3000.0], (0.0,), 20.0),
])
def test_scipy_pair_matches_oracle(nt, nx, v, t0, fp):
    g = stolt.Geometry(nt, nx, DT, DX, v, t0s=t0, wavelet_peak_hz=fp)
    rng = np.random.default_rng(5)
    m = rng.standard_normal(g.model_shape)
    d = rng.standard_normal(g.data_shape)
    ref_d, ref_m = stolt.forward(g, m), stolt.adjoint(g, d)
    for dtype, tol in (("float64", 1e-10), ("float32", 1e-4)):
        op = bench.ScipyStolt(nt, nx, DT, DX, v, t0s=t0, wavelet_peak_hz=fp, dtype=dtype,
                              workers=2)
        assert (op.Nt, op.Nx) == (g.Nt, g.Nx)
        fd = op.forward(m)
        am = op.adjoint(d, len(t0), len(v))
        assert np.linalg.norm(fd - ref_d) / np.linalg.norm(ref_d) < tol, dtype
        assert np.linalg.norm(am - ref_m) / np.linalg.norm(ref_m) < tol, dtype
