"""Own radix-2 FFT for the oracle (test infrastructure only).

Convention (Section 3.2, Fourier coefficients and basis T_pq): the forward
transform is unnormalised,
    phat_k = sum_m phi_m exp(-2 pi i k m / N),
and the inverse carries the 1/N factor,
    phi_m = (1/N) sum_k phat_k exp(+2 pi i k m / N).
(The paper writes the basis as exp(i v_p (x_m + L)) with v_p = pi p / L and
h = 2L/N, i.e. exp(2 pi i p m / N); coefficient p lives at index k = p mod N.
The paper's reconstruction formula omits the 1/N^d factor; the inverse here
includes it.)

Algorithm: iterative decimation-in-time Cooley-Tukey on bit-reversed input,
vectorised over all other axes.  N must be a power of two.
"""
from __future__ import annotations

import numpy as np


def _bitrev(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft_axis(a: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """1-D DFT of `a` along `axis` (returns a new complex128 array)."""
    a = np.asarray(a, dtype=np.complex128)
    x = np.moveaxis(a, axis, -1)
    n = x.shape[-1]
    if n < 1 or (n & (n - 1)) != 0:
        raise ValueError(f"FFT length {n} is not a power of two")
    x = x[..., _bitrev(n)].copy()
    lead = x.shape[:-1]
    sign = 1.0 if inverse else -1.0
    m = 1
    while m < n:
        w = np.exp(sign * 1j * np.pi * np.arange(m) / m)  # exp(-+2 pi i j / (2m))
        y = x.reshape(lead + (n // (2 * m), 2, m))
        even = y[..., 0, :]
        odd = y[..., 1, :] * w
        out = np.empty_like(y)
        out[..., 0, :] = even + odd
        out[..., 1, :] = even - odd
        x = out.reshape(lead + (n,))
        m *= 2
    if inverse:
        x = x / n
    return np.moveaxis(x, -1, axis)


def fftn(a: np.ndarray, axes) -> np.ndarray:
    """Forward transform over each of `axes` in turn."""
    for ax in axes:
        a = fft_axis(a, ax, inverse=False)
    return a


def ifftn(a: np.ndarray, axes) -> np.ndarray:
    """Inverse transform (with 1/N per axis) over each of `axes` in turn."""
    for ax in axes:
        a = fft_axis(a, ax, inverse=True)
    return a


def dft_bruteforce(a: np.ndarray, inverse: bool = False) -> np.ndarray:
    """O(N^2) DFT of a 1-D array, straight from the definition (for pinning)."""
    a = np.asarray(a, dtype=np.complex128)
    n = a.shape[0]
    k = np.arange(n)
    sign = 1.0 if inverse else -1.0
    mat = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
    out = mat @ a
    return out / n if inverse else out
