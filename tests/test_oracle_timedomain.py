"""Pins for the time-domain ASHRT/AASHRT oracle (ch. 3 Table, ch. 6 Eqs
ch6_AASHRT_forward / ch6_AASHRT_adjoint)."""
import numpy as np
import pytest
from scipy.signal import hilbert

from oracle import stolt, timedomain
from paper_1711_10214_gb300 import synth

DT, DX = 0.004, 12.5


def test_dot_product():
    rng = np.random.default_rng(0)
    nt, nx, v, t0 = 40, 10, [1500.0, 2600.0], [0.0, 0.03]
    m = rng.standard_normal((2, 2, nx, nt))
    d = rng.standard_normal((nx, nt))
    Lm = timedomain.forward(nt, nx, DT, DX, v, m, t0)
    LTd = timedomain.adjoint(nt, nx, DT, DX, v, d, t0)
    assert abs(np.vdot(Lm, d) - np.vdot(m, LTd)) / (np.linalg.norm(Lm) * np.linalg.norm(d)) < 1e-13


def test_spike_lands_on_sample_when_exact():
    """A model spike whose path hits a sample exactly puts all of its weight
    there: apex trace, t = tau0 + tau."""
    nt, nx, dt = 32, 5, 1.0 / 256.0     # 3 dt exact in float32
    m = np.zeros((1, 1, nx, nt))
    m[0, 0, 2, 10] = 1.0
    d = timedomain.forward(nt, nx, dt, DX, [2000.0], m, [3 * dt])
    assert d[2, 13] == 1.0 and np.count_nonzero(d[2]) == 1


def test_time_domain_and_stolt_agree_kinematically():
    """Both operators put a model wavelet on the same hyperbola."""
    nt, nx, v, tau, a = 256, 48, 2200.0, 0.35, 24
    m = np.zeros((1, 1, nx, nt))
    m[0, 0, a] = synth.ricker(np.arange(nt) * DT - tau, 20.0)
    d_td = timedomain.forward(nt, nx, DT, DX, [v], m)
    d_st = stolt.forward(stolt.Geometry(nt, nx, DT, DX, [v]), m)
    x = np.arange(nx) * DX
    tc = np.sqrt(tau ** 2 + ((x - a * DX) / v) ** 2)
    ok = np.abs(x - a * DX) / (v * tc) < np.sin(np.pi / 3)
    for d in (d_td, d_st):
        env = np.abs(hilbert(d, axis=1))
        for j in np.nonzero(ok)[0]:
            lo, hi = int((tc[j] - 0.06) / DT), int((tc[j] + 0.06) / DT)
            pk = lo + np.argmax(env[j, lo:hi + 1])
            assert abs(pk - np.rint(tc[j] / DT)) <= 2


def test_domain_of_the_time_domain_pair():
    """v > 0 and tau0 >= 0 (the GPU entry points refuse the same inputs)."""
    m = np.zeros((1, 1, 4, 16))
    with pytest.raises(ValueError):
        timedomain.forward(16, 4, DT, DX, [0.0], m)
    with pytest.raises(ValueError):
        timedomain.adjoint(16, 4, DT, DX, [1500.0], np.zeros((4, 16)), [-0.01])
