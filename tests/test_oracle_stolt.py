"""Pins for the Stolt ASHRT/AASHRT oracle (ch. 5 and ch. 6 operator pairs).

Each pin checks the oracle against something other than itself: the
transpose identity, closed-form special cases (v = 0, laterally constant
models, integer-sample asymptote shifts), exact linear-interpolation values,
the slope bound of the dispersion relation (at most one source of each kind
per output bin), and the analytic traveltime curve of ch. 3 Table
ch3_table_Radon_operators.
"""
import numpy as np
import pytest
from scipy.signal import hilbert

from oracle import stolt
from paper_1711_10214_gb300 import synth

DT, DX = 0.004, 12.5


def _dot_rel(g, rng, mask=None):
    m = rng.standard_normal(g.model_shape)
    d = rng.standard_normal(g.data_shape)
    Lm = stolt.forward(g, m, mask)
    LTd = stolt.adjoint(g, d, mask)
    return abs(np.vdot(Lm, d) - np.vdot(m, LTd)) / (np.linalg.norm(Lm) * np.linalg.norm(d))


@pytest.mark.parametrize("kw", [
    dict(nt=64, nx=16, velocities=[1500.0, 2500.0]),
    dict(nt=50, nx=13, velocities=[1800.0], Nt=128, Nx=32),
    dict(nt=64, nx=16, velocities=[1500.0, 3000.0], t0s=[0.0, 0.05, 0.13]),
    dict(nt=64, nx=16, velocities=[2000.0], wavelet_peak_hz=25.0, fmax_hz=80.0),
])
def test_dot_product(kw):
    kw = dict(kw)
    g = stolt.Geometry(kw.pop("nt"), kw.pop("nx"), DT, DX, kw.pop("velocities"), **kw)
    rng = np.random.default_rng(1)
    assert _dot_rel(g, rng) < 1e-12
    mask = (rng.random(g.nx) < 0.5).astype(float)
    assert _dot_rel(g, rng, mask) < 1e-12


def _remove_w_nyquist(x, Nt, Nx):
    """x padded to (Nx, Nt), its w = 0 and w-Nyquist columns removed, cropped
    (numpy FFT).  With a = 0 the strict cone rule k^2 > a^2 excludes k = 0."""
    nx, nt = x.shape
    X = np.fft.fft2(np.pad(x, ((0, Nx - nx), (0, Nt - nt))))
    X[:, Nt // 2] = 0
    X[:, 0] = 0
    return np.real(np.fft.ifft2(X))[:nx, :nt]


def test_zero_velocity_is_identity():
    """v = 0: a = 0, u = k, the map is the identity; only the w = 0 and
    w-Nyquist bins (excluded by the cone rule) are lost."""
    rng = np.random.default_rng(2)
    g = stolt.Geometry(40, 12, DT, DX, [0.0])
    m = rng.standard_normal(g.model_shape)
    d = stolt.forward(g, m)
    np.testing.assert_allclose(d, _remove_w_nyquist(m[0, 0], g.Nt, g.Nx), atol=1e-12)


def test_laterally_constant_model_sums_panels():
    """Without x padding a laterally constant model has only k_x = 0, where the
    map is the identity for every v: d = sum over velocities (S of Eq.
    ch5_forward_operator)."""
    rng = np.random.default_rng(5)
    nt, nx = 48, 16
    g = stolt.Geometry(nt, nx, DT, DX, [1500.0, 2200.0, 3100.0], Nx=nx)
    f = rng.standard_normal((3, nt))
    m = np.broadcast_to(f[None, :, None, :], g.model_shape).copy()
    d = stolt.forward(g, m)
    ref = _remove_w_nyquist(np.broadcast_to(f.sum(0), (nx, nt)), g.Nt, nx)
    np.testing.assert_allclose(d, ref, atol=1e-12)


def test_integer_asymptote_shift_is_circular_shift():
    """AASHRT with tau0 = j dt equals the tau0 = 0 output circularly delayed by
    j samples in the padded domain (T of Eq. ch6_forward_operator)."""
    rng = np.random.default_rng(6)
    dt = 1.0 / 256.0            # j * dt exact in float32, as the shifts are rounded to it
    g0 = stolt.Geometry(32, 8, dt, DX, [2000.0])
    j = 7
    gj = stolt.Geometry(32, 8, dt, DX, [2000.0], t0s=[j * dt])
    m = rng.standard_normal(g0.model_shape)
    p0 = stolt.forward(g0, m, padded=True)
    pj = stolt.forward(gj, m, padded=True)
    np.testing.assert_allclose(pj, np.roll(p0, j, axis=1), atol=1e-12)


def test_zero_shift_aashrt_equals_ashrt_and_additivity():
    rng = np.random.default_rng(7)
    vs = [1600.0, 2400.0]
    gA = stolt.Geometry(32, 8, DT, DX, vs, t0s=[0.0, 0.0])
    g = stolt.Geometry(32, 8, DT, DX, vs)
    g1 = stolt.Geometry(32, 8, DT, DX, vs[:1])
    g2 = stolt.Geometry(32, 8, DT, DX, vs[1:])
    m = rng.standard_normal(g.model_shape)
    mA = np.concatenate([m, 2.0 * m], axis=0)
    np.testing.assert_allclose(stolt.forward(gA, mA), 3.0 * stolt.forward(g, m), atol=1e-12)
    np.testing.assert_allclose(stolt.forward(g, m),
                               stolt.forward(g1, m[:, :1]) + stolt.forward(g2, m[:, 1:]),
                               atol=1e-12)


def test_map_is_exact_linear_interpolation_of_u():
    """For a spectrum linear in k, the map returns alpha + beta u with
    u = sgn(k) sqrt(k^2 - a^2) (dispersion relation of ch. 5); outside the
    cone (k^2 <= a^2) it returns 0."""
    g = stolt.Geometry(64, 16, DT, DX, [1700.0])
    kk = np.arange(g.Nt)
    kk = np.where(kk <= g.Nt // 2, kk, kk - g.Nt).astype(float)
    alpha, beta = 0.3, 0.7
    M = np.broadcast_to(alpha + beta * kk, (g.Nx, g.Nt)).astype(complex)
    V = g.map_forward(M, 0)
    for l in (0, 1, 3, 8, 15):
        ll = min(l, g.Nx - l)
        a = 1700.0 * ll * g.Nt * DT / (g.Nx * DX)
        for k in (1, 5, 20, 40, 63, -2, -30, -63):
            idx = k % g.Nt
            if k * k > a * a:
                u = np.sign(k) * np.sqrt(k * k - a * a)
                assert abs(V[l, idx] - (alpha + beta * u)) < 1e-9, (l, k)
            else:
                assert V[l, idx] == 0.0


@pytest.mark.parametrize("nt,nx,v", [
    (1024, 256, synth.velocity_scan(1400.0, 3500.0, 32)),     # the benchmark geometry
    (64, 16, [0.0, 900.0, 1700.0, 5000.0]),
    (300, 37, [1234.5, 2999.0]),
])
def test_each_bin_has_at_most_one_source_of_each_kind(nt, nx, v):
    """u(k + 1) - u(k) = (2k + 1) / (u(k + 1) + u(k)) >= 1 because u(k) <= k:
    on each side of the spectrum the floor tap of consecutive mapped bins
    strictly increases, so every output bin receives at most one primary
    (weight 1 - f) and one secondary (weight f) contribution.  The GPU
    adjoint's source table depends on this; here it is checked on the
    oracle's own FP64 taps, row by row."""
    g = stolt.Geometry(nt, nx, DT, DX, v)
    H = g.Nt // 2
    kk = np.arange(g.Nt)
    kk = np.where(kk <= H, kk, kk - g.Nt)
    for iv in range(len(v)):
        rows, i0, i1, w0, w1, incone = g._taps[iv]
        u = np.where(incone, np.sign(kk) * np.sqrt(np.maximum(
            kk.astype(float) ** 2 - g.cone_a(float(g.v[iv]))[:, None] ** 2, 0.0)), 0.0)
        for l in range(g.Nx):
            for side in (kk > 0, kk < 0):
                sel = incone[l] & side
                if not sel.any():
                    continue
                uu = np.abs(u[l][sel])
                order = np.argsort(np.abs(kk[sel]))
                assert np.all(np.diff(uu[order]) >= 1.0 - 1e-12), (iv, l)
                assert np.all(np.diff(np.floor(uu[order])) >= 1), (iv, l)
                assert len(np.unique(i0[l][sel])) == sel.sum()
                assert len(np.unique(i1[l][sel])) == sel.sum()


def _win_peak(d, tc, w):
    env = np.abs(hilbert(d, axis=1))
    nt = d.shape[1]
    out = np.empty(d.shape[0])
    for j in range(d.shape[0]):
        lo = int(max(0, (tc[j] - w) / DT))
        hi = int(min(nt - 1, (tc[j] + w) / DT))
        out[j] = (lo + np.argmax(env[j, lo:hi + 1])) * DT
    return out


@pytest.mark.parametrize("v,tau,a,t0", [(2000.0, 0.4, 32, 0.0), (1500.0, 0.3, 20, 0.0),
                                        (2500.0, 0.25, 40, 0.12)])
def test_impulse_lies_on_hyperbola(v, tau, a, t0):
    """A model wavelet at (tau, v, x_a, tau0) maps onto t = tau0 + sqrt(tau^2 +
    (x - x_a)^2 / v^2) (ch. 3 Table ch3_table_Radon_operators, AASHRT row):
    the envelope peak near the curve is within 2 samples of it on every
    trace with propagation angle below 60 degrees."""
    nt, nx = 256, 64
    g = stolt.Geometry(nt, nx, DT, DX, [v], t0s=[t0])
    m = np.zeros(g.model_shape)
    m[0, 0, a] = synth.ricker(np.arange(nt) * DT - tau, 20.0)
    d = stolt.forward(g, m)
    x = np.arange(nx) * DX
    tc = t0 + np.sqrt(tau ** 2 + ((x - a * DX) / v) ** 2)
    sin_angle = np.abs(x - a * DX) / (v * (tc - t0))
    ok = sin_angle < np.sin(np.pi / 3)
    pk = _win_peak(d, tc, 0.06)
    assert np.max(np.abs(np.rint(pk / DT) - np.rint(tc / DT))[ok]) <= 2
    # the wrong velocity convention (v/2) puts the far traces well off the curve
    tc_half = t0 + np.sqrt(tau ** 2 + (2 * (x - a * DX) / v) ** 2)
    far = ok & (np.abs(tc_half - tc) > 10 * DT)
    if far.any():
        assert np.all(np.abs(pk - tc_half)[far] > 4 * DT)


def test_adjoint_of_data_event_focuses_at_apex():
    """The adjoint of a data hyperbola t = sqrt(tau^2 + (x-x_a)^2/v^2) focuses
    at (tau, v, x_a): the model energy peak is at that apex (Eq. ch5_Stolt_adj)."""
    nt, nx, v, tau, a = 256, 64, 2000.0, 0.5, 30
    g = stolt.Geometry(nt, nx, DT, DX, [1500.0, 2000.0, 2500.0])
    ev = dict(tau=np.array([tau]), xa=np.array([a * DX]), v=np.array([v]),
              A=np.array([1.0]), t0=np.zeros(1))
    d = synth.render(ev, nt, nx, DT, DX, 20.0)
    m = stolt.adjoint(g, d)
    env = np.abs(hilbert(m, axis=-1))
    j, i, xa, it = np.unravel_index(np.argmax(env), env.shape)
    assert i == 1 and abs(xa - a) <= 1 and abs(it * DT - tau) <= 2 * DT


def _ricker_spectrum(f, f_peak, dt):
    """Amplitude spectrum of the generator's sampled Ricker wavelet at the
    frequencies f: the discrete-time Fourier transform of synth.ricker on a
    symmetric window of +-10/f_peak (the wavelet is even, so the transform
    is a cosine sum).  Independent of the oracle's closed form."""
    n = int(np.ceil(10.0 / (f_peak * dt)))
    t = np.arange(-n, n + 1) * dt
    r = synth.ricker(t, f_peak)
    return np.abs(np.cos(2.0 * np.pi * np.outer(np.atleast_1d(f), t)) @ r) * dt


@pytest.mark.parametrize("Nt,dt,fp", [(1000, 0.004, 25.0), (2048, 0.004, 25.0),
                                      (512, 0.004, 20.0), (4096, 0.002, 30.0),
                                      (256, 0.008, 8.0)])
def test_spectral_weight_is_the_ricker_amplitude_spectrum(Nt, dt, fp):
    """The wavelet C of ch. 4 ("a zero phase wavelet with an amplitude
    spectrum similar to ... the data"): Geometry.W must equal the amplitude
    spectrum of the Ricker wavelet the generator renders, normalised to 1 at
    its peak frequency, on every bin of the padded grid; the w-Nyquist bin is
    0 and the zero-frequency bin is 0.  The spectrum is computed numerically
    from the sampled wavelet, so a wrong exponent, a missing square or a
    different normalisation in the oracle fails here."""
    g = stolt.Geometry(Nt // 4, 8, dt, 12.5, [1500.0], Nt=Nt, Nx=16, wavelet_peak_hz=fp)
    kk = np.arange(Nt)
    kk = np.where(kk <= Nt // 2, kk, kk - Nt)
    f = np.abs(kk) / (Nt * dt)
    ref = _ricker_spectrum(f, fp, dt) / _ricker_spectrum(fp, fp, dt)
    ref[Nt // 2] = 0.0
    np.testing.assert_allclose(g.W, ref, rtol=0, atol=2e-9)
    assert g.W[0] == 0.0 and g.W[Nt // 2] == 0.0
    if Nt == 1000:                      # 25 Hz is bin 100 of a 0.25 Hz grid: W = 1 exactly
        assert g.W[100] == pytest.approx(1.0, abs=1e-15)
        assert g.W[Nt - 100] == pytest.approx(1.0, abs=1e-15)
    assert np.all(g.W <= 1.0 + 1e-15)
    # without the wavelet W is 1 except at the Nyquist bin
    g0 = stolt.Geometry(Nt // 4, 8, dt, 12.5, [1500.0], Nt=Nt, Nx=16)
    assert np.all(np.delete(g0.W, Nt // 2) == 1.0) and g0.W[Nt // 2] == 0.0


def test_band_limit_edge():
    """fmax (ch. 5: the map runs over "a limited group of positive
    frequencies"): |f| > fmax is zeroed in both directions, |f| = fmax and
    below are kept unchanged.  dt 4 ms, Nt 1000: bins are 0.25 Hz apart, so
    fmax = 50 Hz is exactly bin 200."""
    Nt, dt = 1000, 0.004
    full = stolt.Geometry(250, 8, dt, 12.5, [1500.0], Nt=Nt, Nx=16, wavelet_peak_hz=25.0)
    lim = stolt.Geometry(250, 8, dt, 12.5, [1500.0], Nt=Nt, Nx=16, wavelet_peak_hz=25.0,
                         fmax_hz=50.0)
    keep = np.r_[0:201, Nt - 200:Nt]
    np.testing.assert_array_equal(lim.W[keep], full.W[keep])
    assert np.all(lim.W[201:Nt - 200] == 0.0)
    assert full.W[201] > 0.1 and full.W[Nt - 201] > 0.1


@pytest.mark.parametrize("Nt,Nx,v", [(256, 64, 2000.0), (512, 32, 1500.0), (512, 128, 3000.0)])
def test_adjoint_carries_the_stolt_jacobian(Nt, Nx, v):
    """ch. 5 Eq. ch5_Stolt_adj: changing the integration variable from w to
    w_tau brings the factor C = w_tau / w into the adjoint.  The exact
    transpose of the linear-interpolation map carries it implicitly: each
    source bin k sends a total weight of 1 to the w_tau bins around
    u(k) = sqrt(k^2 - a^2), and the sources are dk/du = u / k = w_tau / w per
    bin.  So the adjoint of a data spike at (t, x) = (0, 0), whose spectrum is
    flat, has the 2-D spectrum C(w_tau, k_x) = w_tau / sqrt(w_tau^2 + a^2)
    when averaged over 32 bins (a sanity pin: single bins fluctuate with the
    interpolation fractions).  Checked on both w sides and both k_x sides,
    away from the cone edge (C >= 0.4) and from the w-Nyquist bin, without
    padding so that nothing is cropped; the spectrum is taken with numpy's
    FFT.  The forward-style gather (C = 1) or an explicit extra C (C^2)
    misses by more than 10% on every such window."""
    g = stolt.Geometry(Nt, Nx, DT, DX, [v], Nt=Nt, Nx=Nx)
    d = np.zeros((Nx, Nt))
    d[0, 0] = 1.0
    S = np.fft.fft2(stolt.adjoint(g, d)[0, 0])
    assert np.max(np.abs(S.imag)) < 1e-12
    S = S.real
    H, w = Nt // 2, 32
    a_all = g.cone_a(v)
    checked = 0
    for l in range(1, Nx // 2):
        a = a_all[l]
        if a >= H - 1:
            continue
        umax = np.sqrt((H - 1) ** 2 - a * a)
        for j0 in range(1, int(umax) - w - 1, w // 2):
            jj = np.arange(j0, j0 + w)
            C = jj / np.sqrt(jj * jj + a * a)
            if C.min() < 0.4:
                continue
            for side in (S[l, jj], S[l, Nt - jj], S[Nx - l, jj]):
                assert abs(side.mean() - C.mean()) <= 0.05 * C.mean(), (l, j0)
                checked += 1
            if C.mean() < 0.85:
                assert abs(1.0 - C.mean()) > 0.1 * C.mean()
    assert checked > 300
