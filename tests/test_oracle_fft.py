"""Pins of the oracle's own DFTs (no GPU)."""
import numpy as np
import pytest

from oracle import fft as offt


SIZES = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 25, 27, 30, 32, 48, 64, 96, 100, 128, 192, 256]


@pytest.mark.parametrize("n", SIZES)
def test_fft_matches_definition_and_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    ref = np.fft.fft(x)  # an independent library routine
    scale = np.abs(ref).max()
    assert np.abs(offt.fft(x) - ref).max() <= 1e-14 * scale * max(1, np.log2(n))
    assert np.abs(offt.dft_direct(x) - ref).max() <= 1e-13 * scale
    assert np.abs(offt.ifft(x) - np.fft.ifft(x)).max() <= 1e-14 * scale
    assert np.abs(offt.dft_direct(x, inverse=True) - np.fft.ifft(x)).max() <= 1e-13 * scale


def test_delta_and_constant():
    n = 24
    e = np.zeros(n, complex)
    e[5] = 1.0
    k = np.arange(n)
    assert np.allclose(offt.fft(e), np.exp(-2j * np.pi * 5 * k / n), atol=1e-15)
    assert np.allclose(offt.fft(np.ones(n)), n * (k == 0), atol=1e-13)


def test_roundtrip_parseval_and_axes():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((6, 10, 12)) + 1j * rng.standard_normal((6, 10, 12))
    X = offt.fftn(x)
    assert np.abs(offt.ifftn(X) - x).max() < 1e-14
    assert np.isclose(np.sum(np.abs(X) ** 2), x.size * np.sum(np.abs(x) ** 2), rtol=1e-13)
    assert np.abs(X - np.fft.fftn(x)).max() < 1e-12
    assert np.abs(offt.fft(x, axis=1) - np.fft.fft(x, axis=1)).max() < 1e-13
