"""Pins for the irregular-trace form of the Stolt oracle (ch. 6: for
non-uniform spatial sampling the x transform becomes a discrete Fourier
transform evaluated at the trace positions).

Checked against: the regular operator at regular positions, numpy's FFT
(trigonometric interpolation of the padded regular field at half-sample
positions), the transpose identity, and the analytic traveltime curve at
irregular offsets."""
import numpy as np
import pytest
from scipy.signal import hilbert

from oracle import stolt
from paper_1711_10214_gb300 import synth

DT, DX = 0.004, 12.5


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_regular_positions_reduce_to_the_regular_operator():
    g = stolt.Geometry(64, 16, DT, DX, [1500.0, 2600.0], t0s=[0.0, 0.05])
    rng = np.random.default_rng(0)
    m = rng.standard_normal(g.model_shape)
    d = rng.standard_normal(g.data_shape)
    x = np.arange(g.nx) * DX
    assert _rel(stolt.forward_irregular(g, m, x), stolt.forward(g, m)) < 1e-12
    assert _rel(stolt.adjoint_irregular(g, d, x), stolt.adjoint(g, d)) < 1e-12


def test_half_sample_positions_are_the_trigonometric_interpolation():
    """At x = (j + 1/2) dx the irregular forward equals the band-limited
    interpolation of the padded regular field, done here with numpy's FFT
    (a half-sample phase ramp, the k_x-Nyquist term split evenly)."""
    g = stolt.Geometry(48, 12, DT, DX, [1800.0])
    rng = np.random.default_rng(1)
    m = rng.standard_normal(g.model_shape)
    F = stolt.forward(g, m, padded=True)                    # [Nx][Nt], periodic in x
    s = np.fft.fftfreq(g.Nx, d=1.0 / g.Nx)                  # signed indices (Nyquist negative)
    ramp = np.exp(2j * np.pi * s * 0.5 / g.Nx)
    ramp[g.Nx // 2] = np.cos(np.pi * 0.5)                   # Nyquist: cos(pi (j + 1/2)) -> 0 at j = 0
    G = np.real(np.fft.ifft(np.fft.fft(F, axis=0) * ramp[:, None], axis=0))
    x = (np.arange(g.nx) + 0.5) * DX
    assert _rel(stolt.forward_irregular(g, m, x), G[:g.nx, :g.nt]) < 1e-10


def test_irregular_pair_is_a_transpose_pair():
    g = stolt.Geometry(64, 16, DT, DX, [1500.0, 2300.0], t0s=[0.0, 0.04],
                       wavelet_peak_hz=25.0)
    rng = np.random.default_rng(2)
    x = np.sort(rng.uniform(0.0, (g.nx - 1) * DX, 11))
    mask = (rng.random(11) < 0.8).astype(float)
    m = rng.standard_normal(g.model_shape)
    d = rng.standard_normal((11, g.nt))
    lhs = np.vdot(stolt.forward_irregular(g, m, x, mask), d)
    rhs = np.vdot(m, stolt.adjoint_irregular(g, d, x, mask))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("v,tau,a", [(2000.0, 0.4, 32), (1500.0, 0.3, 20)])
def test_impulse_lies_on_the_hyperbola_at_irregular_offsets(v, tau, a):
    nt, nx = 256, 64
    g = stolt.Geometry(nt, nx, DT, DX, [v])
    m = np.zeros(g.model_shape)
    m[0, 0, a] = synth.ricker(np.arange(nt) * DT - tau, 20.0)
    x = np.sort(np.random.default_rng(3).uniform(0.0, (nx - 1) * DX, 40))
    d = stolt.forward_irregular(g, m, x)
    tc = np.sqrt(tau ** 2 + ((x - a * DX) / v) ** 2)
    ok = np.abs(x - a * DX) / (v * tc) < np.sin(np.pi / 3)
    env = np.abs(hilbert(d, axis=1))
    for j in np.nonzero(ok)[0]:
        lo = int(max(0, (tc[j] - 0.06) / DT))
        hi = int(min(nt - 1, (tc[j] + 0.06) / DT))
        pk = lo + np.argmax(env[j, lo:hi + 1])
        assert abs(pk - np.rint(tc[j] / DT)) <= 2, (j, x[j])
