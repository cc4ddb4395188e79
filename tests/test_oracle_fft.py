"""Pins of the oracle FFT: brute-force DFT from the definition (Section 3.2),
numpy's FFT as an independent library routine, round trips."""
import numpy as np
import pytest

from oracle.fft import dft_bruteforce, fft_axis, fftn, ifftn


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32])
def test_fft_matches_bruteforce_dft(n):
    rng = np.random.default_rng(n)
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    np.testing.assert_allclose(fft_axis(a, 0), dft_bruteforce(a), atol=1e-13 * max(1, n))
    np.testing.assert_allclose(fft_axis(a, 0, inverse=True), dft_bruteforce(a, inverse=True), atol=1e-14 * max(1, n))


@pytest.mark.parametrize("n", [64, 128, 512])
def test_fft_matches_numpy(n):
    rng = np.random.default_rng(7)
    a = rng.normal(size=(3, n)) + 1j * rng.normal(size=(3, n))
    np.testing.assert_allclose(fft_axis(a, -1), np.fft.fft(a, axis=-1), atol=1e-12 * n)
    np.testing.assert_allclose(fft_axis(a, -1, inverse=True), np.fft.ifft(a, axis=-1), atol=1e-14 * n)


def test_fft_other_axis_and_nd():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(3, 8, 16, 32)) + 1j * rng.normal(size=(3, 8, 16, 32))
    np.testing.assert_allclose(fft_axis(a, 1), np.fft.fft(a, axis=1), atol=1e-11)
    np.testing.assert_allclose(fftn(a, (-1, -2, -3)), np.fft.fftn(a, axes=(-1, -2, -3)), atol=1e-10)
    np.testing.assert_allclose(ifftn(fftn(a, (-1, -2)), (-1, -2)), a, atol=1e-13)


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        fft_axis(np.zeros(12, complex), 0)


def test_single_mode_exact():
    # exp(2 pi i k0 m / N) transforms to N * delta_{k,k0} (definition of the DFT)
    n, k0 = 32, 5
    m = np.arange(n)
    a = np.exp(2j * np.pi * k0 * m / n)
    out = fft_axis(a, 0)
    expect = np.zeros(n, complex)
    expect[k0] = n
    np.testing.assert_allclose(out, expect, atol=1e-12)
