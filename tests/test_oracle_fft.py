"""Pins for the oracle's FFT: the O(N^2) textbook sum, exact single modes,
Parseval, the inverse, and numpy's independent pocketfft."""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(1601)


def _rand(n):
    return RNG.standard_normal(n) + 1j * RNG.standard_normal(n)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 7, 11])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_direct_sum(n, sign):
    x = _rand(n)
    # textbook sum written here independently of the oracle
    j = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    ref = W @ x
    assert np.allclose(oracle.fft(x, sign), ref, rtol=0, atol=1e-12 * max(1, n))
    assert np.allclose(oracle.dft(x, sign), ref, rtol=0, atol=1e-12 * max(1, n))


@pytest.mark.parametrize("n", [32, 64, 96, 128, 160, 256, 384, 512])
def test_fft_matches_numpy(n):
    x = _rand(n)
    assert np.max(np.abs(oracle.fft(x, -1) - np.fft.fft(x))) < 1e-12 * n
    assert np.max(np.abs(oracle.fft(x, 1) - np.fft.ifft(x) * n)) < 1e-12 * n


@pytest.mark.parametrize("n,m", [(64, 3), (96, 7), (160, 80), (256, 1)])
def test_single_mode(n, m):
    j = np.arange(n)
    x = np.exp(2j * np.pi * m * j / n)
    X = oracle.fft(x, -1)
    ref = np.zeros(n, complex)
    ref[m] = n
    assert np.max(np.abs(X - ref)) < 1e-11


@pytest.mark.parametrize("n", [60, 120, 250])
def test_parseval_and_roundtrip(n):
    x = _rand(n)
    X = oracle.fft(x, -1)
    assert abs(np.sum(np.abs(X) ** 2) / n - np.sum(np.abs(x) ** 2)) < 1e-10 * n
    assert np.max(np.abs(oracle.fft(X, 1) / n - x)) < 1e-13 * n


def test_fftn_matches_numpy():
    a = RNG.standard_normal((6, 10, 12)) + 1j * RNG.standard_normal((6, 10, 12))
    assert np.max(np.abs(oracle.fftn(a, -1) - np.fft.fftn(a))) < 1e-11
    assert np.max(np.abs(oracle.fftn(a, 1) - np.fft.ifftn(a) * a.size)) < 1e-11
