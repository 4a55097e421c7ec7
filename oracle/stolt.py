"""Stolt-based ASHRT and AASHRT, forward and exact transpose, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows the operator factorisations of the thesis:
  ch. 5 Eq. ch5_forward_operator   L  = S F^{-1} M F          (sum over v)
  ch. 5 Eq. ch5_adj_operator       L^T = F^{-1} M^T F S^T     (spray over v)
  ch. 6 Eq. ch6_forward_operator   L  = S A F^{-1} T M F      (sum over v, tau0;
                                                              T = exp(-i w tau0))
  ch. 6 Eq. ch6_adj_operator       L^T = F^{-1} M^T T^T F A^T S^T
with the Stolt dispersion relation w_tau = sqrt(w^2 - (v k_x)^2) (ch. 5 and
ch. 6, "modified dispersion relationship") and, optionally, the zero-phase
wavelet C of ch. 4 ("L replaced by C L").

Readings taken where the thesis is silent or inconsistent:
  * analysis exp(-i), synthesis exp(+i); velocity enters as v (not v/2);
  * the T shift acts on the data frequency w: forward exp(-i w tau0);
  * M is 2-tap linear interpolation along w at fixed k_x; the adjoint is the
    exact transpose of the forward (the change-of-variables factor C of
    Eq. ch5_Stolt_adj is then carried implicitly by the transpose);
  * a bin (k, l) is mapped iff k^2 > a^2 strictly and k is not the w-Nyquist
    bin, with a = ((v*|l|)*Nt)*dt / (Nx*dx) evaluated in IEEE double in
    exactly that order (the w_tau index is u = sgn(k) sqrt(k^2 - a^2));
  * a tap that lands on the w-Nyquist bin reads (and, transposed, writes) 0;
  * zero padding nt -> Nt, nx -> Nx (default: next power of two >= 2n);
  * optional band limit and Ricker amplitude spectrum are part of W(w).
"""
import numpy as np

from . import dft as _dft


def next_pow2(n):
    p = 1
    while p < n:
        p *= 2
    return p


class Geometry:
    """Grids and scan parameters of one Stolt ASHRT/AASHRT operator.

    velocities and t0 shifts are rounded to float32 first: the CUDA library
    receives them as float32, so both sides scan the same parameters.
    Model layout: m[nt0][nv][nx][nt]; data layout: d[nx][nt].
    """

    def __init__(self, nt, nx, dt, dx, velocities, t0s=(0.0,), Nt=None, Nx=None,
                 pad_t=2, pad_x=2, fmax_hz=0.0, wavelet_peak_hz=0.0):
        self.nt, self.nx = int(nt), int(nx)
        self.dt, self.dx = float(dt), float(dx)
        self.v = np.asarray(velocities, dtype=np.float32).astype(np.float64).ravel()
        self.t0 = np.asarray(t0s, dtype=np.float32).astype(np.float64).ravel()
        self.Nt = int(Nt) if Nt is not None else next_pow2(pad_t * self.nt)
        self.Nx = int(Nx) if Nx is not None else next_pow2(pad_x * self.nx)
        assert self.Nt >= self.nt and self.Nx >= self.nx and self.Nt % 2 == 0
        self.nv, self.nt0 = len(self.v), len(self.t0)
        self.fmax_hz = float(fmax_hz)
        self.wavelet_peak_hz = float(wavelet_peak_hz)
        self._taps = [self._stolt_taps(v) for v in self.v]
        self.W = self._spectral_weight()
        kk = _dft.signed_index(self.Nt).astype(np.float64)
        # T of Eq. ch6_forward_operator: exp(-i w tau0), w = 2 pi k / (Nt dt)
        self.phase = [np.exp(-2j * np.pi * kk * t0 / (self.Nt * self.dt)) for t0 in self.t0]

    @property
    def model_shape(self):
        return (self.nt0, self.nv, self.nx, self.nt)

    @property
    def data_shape(self):
        return (self.nx, self.nt)

    # -- Stolt map M (ch. 5 Eqs ch5_Stolt_adj / ch5_Stolt_forward) ----------
    def cone_a(self, v):
        """a_l = v |k_x| / dw in w-bin units, evaluated as ((v*|l|)*Nt)*dt/(Nx*dx)."""
        labs = np.abs(_dft.signed_index(self.Nx)).astype(np.float64)
        return ((v * labs) * float(self.Nt)) * self.dt / (float(self.Nx) * self.dx)

    def _stolt_taps(self, v):
        Nt = self.Nt
        kk = _dft.signed_index(Nt).astype(np.float64)[None, :]         # (1, Nt)
        a = self.cone_a(v)[:, None]                                     # (Nx, 1)
        a2 = a * a
        incone = (kk * kk > a2) & (kk != Nt // 2)
        u = np.where(incone, np.sign(kk) * np.sqrt(np.maximum(kk * kk - a2, 0.0)), 0.0)
        k0 = np.floor(u)
        f = u - k0
        k0 = k0.astype(np.int64)
        i0 = np.mod(k0, Nt)
        i1 = np.mod(k0 + 1, Nt)
        w0 = np.where(incone, 1.0 - f, 0.0)
        w1 = np.where(incone, f, 0.0)
        # a tap on the w-Nyquist bin reads 0
        w0 = np.where(i0 == Nt // 2, 0.0, w0)
        w1 = np.where(i1 == Nt // 2, 0.0, w1)
        rows = np.broadcast_to(np.arange(self.Nx)[:, None], i0.shape)
        return rows, i0, i1, w0, w1, incone

    def map_forward(self, Mhat, iv):
        """V(k, l) = (1-f) Mhat(k0, l) + f Mhat(k0+1, l) inside the cone, else 0."""
        rows, i0, i1, w0, w1, _ = self._taps[iv]
        return w0 * Mhat[rows, i0] + w1 * Mhat[rows, i1]

    def map_adjoint(self, D, iv):
        """Exact transpose of map_forward: scatter D(k, l) to the two taps."""
        rows, i0, i1, w0, w1, _ = self._taps[iv]
        out = np.zeros_like(D)
        np.add.at(out, (rows, i0), w0 * D)
        np.add.at(out, (rows, i1), w1 * D)
        return out

    # -- W(w): wavelet C (ch. 4), band limit, Nyquist ----------------------
    def _spectral_weight(self):
        kk = _dft.signed_index(self.Nt).astype(np.float64)
        f = np.abs(kk) / (self.Nt * self.dt)
        W = np.ones(self.Nt)
        if self.wavelet_peak_hz > 0.0:
            z = (f / self.wavelet_peak_hz) ** 2
            W = z * np.exp(1.0 - z)          # Ricker amplitude spectrum, max 1
        if self.fmax_hz > 0.0:
            W = np.where(f > self.fmax_hz, 0.0, W)
        W[self.Nt // 2] = 0.0
        return W


def forward(g, m, mask=None, padded=False):
    """d = S C F^{-1} sum_{tau0} T sum_v M F m   (Eqs ch5/ch6_forward_operator).

    m: model [nt0][nv][nx][nt]; mask: per-trace weights [nx] (sampling S) or
    None.  Returns d [nx][nt] (or the uncropped [Nx][Nt] field if padded).
    """
    m = np.asarray(m, dtype=np.float64).reshape(g.model_shape)
    N = g.Nt * g.Nx
    D = np.zeros((g.Nx, g.Nt), dtype=np.complex128)
    for j in range(g.nt0):
        Dj = np.zeros_like(D)
        for i in range(g.nv):
            Dj += g.map_forward(_dft.dft2(m[j, i], g.Nx, g.Nt), i)
        D += g.phase[j][None, :] * Dj
    D *= g.W[None, :]
    if padded:
        return np.real(_dft.idft2_unnormalised(D, g.Nx, g.Nt)) / N
    d = np.real(_dft.idft2_unnormalised(D, g.nx, g.nt)) / N
    if mask is not None:
        d = d * np.asarray(mask, dtype=np.float64)[:, None]
    return d


def adjoint(g, d, mask=None):
    """m = F^{-1} M^T T^T F A^T S^T d : the exact transpose of ``forward``."""
    d = np.asarray(d, dtype=np.float64).reshape(g.data_shape)
    if mask is not None:
        d = d * np.asarray(mask, dtype=np.float64)[:, None]
    N = g.Nt * g.Nx
    Dh = _dft.dft2(d, g.Nx, g.Nt) * (g.W[None, :] / N)
    m = np.zeros(g.model_shape)
    for j in range(g.nt0):
        Dj = np.conj(g.phase[j])[None, :] * Dh
        for i in range(g.nv):
            M = g.map_adjoint(Dj, i)
            m[j, i] = np.real(_dft.idft2_unnormalised(M, g.nx, g.nt))
    return m


def forward_batch(g, m, mask=None):
    """forward over a leading batch axis: m [B][nt0][nv][nx][nt] -> [B][nx][nt]."""
    m = np.asarray(m, dtype=np.float64)
    return np.stack([forward(g, m[b], None if mask is None else mask[b])
                     for b in range(m.shape[0])])


def adjoint_batch(g, d, mask=None):
    d = np.asarray(d, dtype=np.float64)
    return np.stack([adjoint(g, d[b], None if mask is None else mask[b])
                     for b in range(d.shape[0])])


# -- irregular trace positions (ch. 6: "the F operator may be replaced by a
#    Discrete Fourier Transform operator" for non-uniform spatial sampling) --
def x_synthesis_matrix(g, x_positions):
    """E[j, l] = exp(+2 pi i s_l x_j / (Nx dx)) for traces at x_j (metres),
    s_l the signed wavenumber index of row l; the k_x-Nyquist row l = Nx/2
    enters as cos(pi x_j / dx), i.e. split evenly between +Nx/2 and -Nx/2
    (reading: symmetric trigonometric interpolation).  At x_j = j dx this is
    the regular synthesis matrix."""
    x = np.asarray(x_positions, dtype=np.float64)[:, None] / (g.Nx * g.dx)
    s = _dft.signed_index(g.Nx).astype(np.float64)[None, :]
    E = np.exp(2j * np.pi * s * x)
    ny = g.Nx // 2
    E[:, ny] = np.cos(np.pi * np.asarray(x_positions, dtype=np.float64) / g.dx)
    return E


def forward_irregular(g, m, x_positions, mask=None):
    """d [nr][nt] at irregular trace positions from a model on the regular
    apex grid: ``forward`` with the x synthesis evaluated at x_positions."""
    m = np.asarray(m, dtype=np.float64).reshape(g.model_shape)
    N = g.Nt * g.Nx
    D = np.zeros((g.Nx, g.Nt), dtype=np.complex128)
    for j in range(g.nt0):
        Dj = np.zeros_like(D)
        for i in range(g.nv):
            Dj += g.map_forward(_dft.dft2(m[j, i], g.Nx, g.Nt), i)
        D += g.phase[j][None, :] * Dj
    D *= g.W[None, :]
    Et = _dft.dft_matrix(g.nt, g.Nt, +1, g.Nt)
    d = np.real(x_synthesis_matrix(g, x_positions) @ D @ Et.T) / N
    if mask is not None:
        d = d * np.asarray(mask, dtype=np.float64)[:, None]
    return d


def adjoint_irregular(g, d, x_positions, mask=None):
    """The exact transpose of ``forward_irregular``: the x analysis of the
    data is the conjugate transpose of the irregular synthesis."""
    d = np.asarray(d, dtype=np.float64)
    if mask is not None:
        d = d * np.asarray(mask, dtype=np.float64)[:, None]
    N = g.Nt * g.Nx
    Ft = _dft.dft_matrix(g.Nt, g.nt, -1, g.Nt)
    Dh = (np.conj(x_synthesis_matrix(g, x_positions)).T @ d @ Ft.T) * (g.W[None, :] / N)
    m = np.zeros(g.model_shape)
    for j in range(g.nt0):
        Dj = np.conj(g.phase[j])[None, :] * Dh
        for i in range(g.nv):
            M = g.map_adjoint(Dj, i)
            m[j, i] = np.real(_dft.idft2_unnormalised(M, g.nx, g.nt))
    return m
