"""Oracle: Fourier conventions and a brute-force DFT.

Test infrastructure only (see ``oracle/__init__.py``).

The paper's FFTs are FFTW (§2.3) and its power spectrum keeps the k_z >= 0 half of a real
transform (§3.3).  Here the 3D transforms are numpy's pocketfft (a library primitive) with the
same layout: real arrays [x, y, z], the half axis is z (the last, fastest axis), forward
X(k) = sum_x x e^{-i k.x}, the inverse carries 1/N^3.  ``naive_dft3`` is the plain O(N^6)
definition written out, used on tiny grids to pin the library transform and the mode order.
"""

from __future__ import annotations

import numpy as np


def mode_numbers(n: int) -> np.ndarray:
    """Signed mode numbers m of a length-n transform in storage order: 0..n/2-1, -n/2..-1."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def half_mode_numbers(n: int) -> np.ndarray:
    """Mode numbers 0..n/2 of the half (real-to-complex) axis."""
    return np.arange(n // 2 + 1, dtype=np.int64)


def mode_grids(n: int):
    """Integer mode grids (mx, my, mz) broadcastable to the half spectrum [n, n, n/2+1]."""
    m = mode_numbers(n)
    mz = half_mode_numbers(n)
    return m[:, None, None], m[None, :, None], mz[None, None, :]


def odd_mode(m: np.ndarray, n: int) -> np.ndarray:
    """m with the Nyquist mode (|m| = n/2) set to 0.

    A single factor i k_j is odd under k -> -k; on the Nyquist plane -k aliases to k, so the
    factor is set to 0 there to keep the inverse transform real (a reading: the paper does not
    state its gradient's Nyquist treatment).
    """
    return np.where(np.abs(m) * 2 == n, 0, m)


def rfft3(x):
    return np.fft.rfftn(np.asarray(x, dtype=np.float64))


def irfft3(xk, n: int):
    return np.fft.irfftn(xk, s=(n, n, n), axes=(0, 1, 2))


def naive_dft3(x) -> np.ndarray:
    """Full complex 3D DFT by the definition X(k) = sum_x x(x) exp(-2 pi i k.x / n), O(n^6)."""
    x = np.asarray(x, dtype=np.complex128)
    n0, n1, n2 = x.shape
    j0, j1, j2 = np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij")
    out = np.empty_like(x)
    for k0 in range(n0):
        for k1 in range(n1):
            for k2 in range(n2):
                ph = -2j * np.pi * (k0 * j0 / n0 + k1 * j1 / n1 + k2 * j2 / n2)
                out[k0, k1, k2] = np.sum(x * np.exp(ph))
    return out
