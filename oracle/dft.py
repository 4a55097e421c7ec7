"""Naive discrete Fourier transforms (the F operators of ch. 5 Eqs
ch5_adj_operator / ch5_forward_operator).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (reading of ch. 5 Eq. ch5_Stolt_adj1 vs ch5_Stolt_forward):
analysis uses exp(-i...), synthesis uses exp(+i...).  A length-``n`` input is
zero-padded to the transform length ``N`` (ch. 5, zero padding for the w-k
interpolation).  Every transform here is the plain definition written as a
matrix product; there is no fast algorithm anywhere in the oracle.
"""
import numpy as np


def dft_matrix(rows, cols, sign, period):
    """E[k, j] = exp(sign * 2*pi*i * k*j / period) for k < rows, j < cols.

    The phase is reduced exactly in integers, (k*j) mod period, before scaling
    so the matrix entries are accurate to one rounding of cos/sin.
    """
    k = np.arange(rows, dtype=np.int64)[:, None]
    j = np.arange(cols, dtype=np.int64)[None, :]
    kj = (k * j) % period
    ang = (2.0 * np.pi / period) * kj.astype(np.float64)
    return np.cos(ang) + (1j * sign) * np.sin(ang)


def dft(x, N):
    """X[k] = sum_{j<n} x[j] exp(-2 pi i k j / N), k < N (zero-padded DFT)."""
    x = np.asarray(x)
    return dft_matrix(N, x.shape[-1], -1, N) @ x


def idft_unnormalised(X, n):
    """x[j] = sum_{k<N} X[k] exp(+2 pi i k j / N) for j < n (cropped)."""
    X = np.asarray(X)
    N = X.shape[-1]
    return dft_matrix(n, N, +1, N) @ X


def dft2(m, Nx, Nt):
    """2-D analysis transform of a gather stored [x][t] (t fastest).

    Mhat[l, k] = sum_{j<nx} sum_{i<nt} m[j, i] exp(-2 pi i (l j / Nx + k i / Nt)).
    Output shape (Nx, Nt): row l = x-wavenumber index, column k = t-frequency.
    """
    m = np.asarray(m)
    nx, nt = m.shape
    Fx = dft_matrix(Nx, nx, -1, Nx)      # (Nx, nx)
    Ft = dft_matrix(Nt, nt, -1, Nt)      # (Nt, nt)
    return Fx @ m @ Ft.T


def idft2_unnormalised(D, nx, nt):
    """2-D synthesis, cropped: d[j, i] = sum_l sum_k D[l, k] exp(+2 pi i (l j/Nx + k i/Nt))."""
    D = np.asarray(D)
    Nx, Nt = D.shape
    Ex = dft_matrix(nx, Nx, +1, Nx)      # (nx, Nx)
    Et = dft_matrix(nt, Nt, +1, Nt)      # (nt, Nt)
    return Ex @ D @ Et.T


def signed_index(N):
    """Signed frequency index of each bin: k for k < N/2, k - N for k > N/2,
    and +N/2 for the Nyquist bin (N even)."""
    k = np.arange(N, dtype=np.int64)
    return np.where(k <= N // 2, k, k - N)
