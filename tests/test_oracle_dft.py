"""Pins for the oracle's naive DFTs (the F operators of ch. 5)."""
import numpy as np
import pytest

from oracle import dft


def test_dft_hand_cases():
    # delta -> all ones; shifted delta -> exp(-2 pi i k / 4) = 1, -i, -1, i
    np.testing.assert_allclose(dft.dft([1, 0, 0, 0], 4), [1, 1, 1, 1], atol=1e-15)
    np.testing.assert_allclose(dft.dft([0, 1, 0, 0], 4), [1, -1j, -1, 1j], atol=1e-15)
    # constant -> N at k=0 only
    np.testing.assert_allclose(dft.dft([1, 1, 1, 1], 4), [4, 0, 0, 0], atol=1e-15)
    # zero padding: [1, 1] padded to 4 -> 1 + exp(-i pi k / 2)
    np.testing.assert_allclose(dft.dft([1, 1], 4), [2, 1 - 1j, 0, 1 + 1j], atol=1e-15)


@pytest.mark.parametrize("n,N", [(5, 8), (16, 16), (7, 32), (33, 64)])
def test_dft_matches_library_fft(n, N):
    rng = np.random.default_rng(n * N)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(dft.dft(x, N), np.fft.fft(x, n=N), rtol=0, atol=1e-12)
    X = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    np.testing.assert_allclose(dft.idft_unnormalised(X, n), (np.fft.ifft(X) * N)[:n], atol=1e-12)


def test_dft2_layout_and_library():
    rng = np.random.default_rng(3)
    m = rng.standard_normal((6, 10))          # [x][t]
    Mh = dft.dft2(m, 8, 16)                    # [l][k]
    ref = np.fft.fft2(np.pad(m, ((0, 2), (0, 6))))
    np.testing.assert_allclose(Mh, ref, atol=1e-12)
    back = dft.idft2_unnormalised(Mh, 6, 10) / (8 * 16)
    np.testing.assert_allclose(back.real, m, atol=1e-12)
    np.testing.assert_allclose(back.imag, 0, atol=1e-12)


def test_parseval():
    rng = np.random.default_rng(4)
    m = rng.standard_normal((8, 16))
    Mh = dft.dft2(m, 8, 16)
    assert abs(np.sum(np.abs(Mh) ** 2) / 128 - np.sum(m * m)) < 1e-10


def test_signed_index():
    assert list(dft.signed_index(8)) == [0, 1, 2, 3, 4, -3, -2, -1]
