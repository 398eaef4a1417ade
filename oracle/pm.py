"""Oracle: particle-mesh force, Poisson solve with the gradient kernel in k space.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages: Poisson equation nabla^2 phi = (3/2) Om a^-1 delta and F = -nabla phi (§2.2,
eq. motion); PM force on a uniform mesh (§2.3; Appendix A).  In mesh-cell units the wavenumber
of mode m is k = 2 pi m / N, so

    F_j(k) = i D(k_j) (3/2)(Om/a) delta(k) / k^2,   k = 0 mode set to 0,

with the continuous Green function -1/k^2 and the gradient kernel of the 4-point central
difference, D(k) = (8 sin k - sin 2k) / 6 (k in radians per cell), which is 0 on the Nyquist
plane.  No deconvolution of the CIC window.  The paper names only "the PM force"; this reading
(not stated in the paper) is the one whose pair force matches Newton beyond ~3 cells with per-cent
scatter (Appendix A), which the continuous i k kernel does not (its point-source force rings at
the mesh scale).
"""

from __future__ import annotations

import numpy as np

from . import cic, fourier


def gradient_kernel(m: np.ndarray, n: int) -> np.ndarray:
    """D(k) = (8 sin k - sin 2k) / 6 at k = 2 pi m / n, exactly 0 on the Nyquist plane."""
    k = 2.0 * np.pi * m.astype(np.float64) / n
    d = (8.0 * np.sin(k) - np.sin(2.0 * k)) / 6.0
    return np.where(np.abs(m) * 2 == n, 0.0, d)


def green_gradient_spectra(delta_k: np.ndarray, n: int, force_scale: float) -> list[np.ndarray]:
    """The three spectra i D(k_j) force_scale delta(k) / k^2 on the half spectrum [n, n, n/2+1]."""
    mx, my, mz = fourier.mode_grids(n)
    kf = 2.0 * np.pi / n
    k2 = (mx * mx + my * my + mz * mz).astype(np.float64) * kf * kf
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(k2 > 0, force_scale / k2, 0.0)
    out = []
    for m in (mx, my, mz):
        out.append(1j * gradient_kernel(m, n) * g * delta_k)
    return out


def force_mesh(delta: np.ndarray, force_scale: float) -> np.ndarray:
    """Force field [3, N, N, N] (mesh-cell units) from the density contrast delta [N, N, N]."""
    n = delta.shape[0]
    dk = fourier.rfft3(delta)
    return np.stack([fourier.irfft3(fk, n) for fk in green_gradient_spectra(dk, n, force_scale)])


def density_fixed(s, np_side: int, nmesh: int) -> np.ndarray:
    """delta on the mesh from the fixed-point deposit of displacements s [3, n]."""
    mesh = cic.cic_fixed_mesh(s, np_side, nmesh)
    return cic.delta_from_fixed(mesh, np_side ** 3)


def pm_force(s, np_side: int, nmesh: int, force_scale: float) -> np.ndarray:
    """Force at each particle [3, n]: deposit, FFT, Green/gradient, inverse FFT, interpolate."""
    fmesh = force_mesh(density_fixed(s, np_side, nmesh), force_scale)
    cell, w1 = cic.interp_weights_fixed(s, np_side, nmesh)
    return cic.cic_interp(fmesh, cell, w1)


# ---- closed forms for a density made of plane waves (checks at mesh sizes too big for an FFT) --------
# delta(x) = sum_w A_w cos(2 pi m_w.x / N + phi_w) on the integer cells x, with every |m_w,i| < N/2
# and m_w != 0.  Its DFT has (A/2) N^3 e^{+i phi} at +m and (A/2) N^3 e^{-i phi} at -m, so the force
# of §2.2 (Green function -1/k^2, gradient kernel D, Poisson prefactor force_scale) is, per wave,
# F_j(x) = -force_scale A D(m_j) sin(2 pi m.x / N + phi) / k^2 with k = 2 pi m / N in rad/cell.

def plane_wave_density(waves, n: int, cells) -> np.ndarray:
    """delta at flat cell indices (ix N + iy) N + iz."""
    cells = np.asarray(cells, dtype=np.int64)
    x = np.stack([cells // (n * n), (cells // n) % n, cells % n]).astype(np.float64)
    out = np.zeros(cells.shape, dtype=np.float64)
    for m, amp, phi in waves:
        theta = 2.0 * np.pi * (m[0] * x[0] + m[1] * x[1] + m[2] * x[2]) / n + phi
        out += amp * np.cos(theta)
    return out


def plane_wave_spectrum(waves, n: int) -> dict:
    """The nonzero entries of the half spectrum [N, N, N/2+1] of the plane-wave density: {(ix, iy, iz):
    complex value} in storage order (negative mode numbers stored at m + N; k_z in 0..N/2)."""
    out = {}
    for m, amp, phi in waves:
        assert 0 < max(abs(int(c)) for c in m) and all(abs(int(c)) * 2 < n for c in m)
        for sign in (+1, -1):
            k = [int(sign * c) % n for c in m]
            if k[2] > n // 2:
                continue   # the conjugate half, not stored
            key = tuple(k)
            out[key] = out.get(key, 0.0) + 0.5 * amp * n ** 3 * np.exp(1j * sign * phi)
    return out


def plane_wave_force(waves, n: int, force_scale: float, cells) -> np.ndarray:
    """Force [3, m] of the plane-wave density at flat cell indices, from the Green function and the
    gradient kernel of ``green_gradient_spectra``."""
    cells = np.asarray(cells, dtype=np.int64)
    x = np.stack([cells // (n * n), (cells // n) % n, cells % n]).astype(np.float64)
    out = np.zeros((3,) + cells.shape, dtype=np.float64)
    kf = 2.0 * np.pi / n
    for m, amp, phi in waves:
        mm = np.asarray(m, dtype=np.int64)
        k2 = float(np.sum(mm * mm)) * kf * kf
        theta = 2.0 * np.pi * (mm[0] * x[0] + mm[1] * x[1] + mm[2] * x[2]) / n + phi
        for j in range(3):
            d = float(gradient_kernel(np.array([mm[j]]), n)[0])
            out[j] += -force_scale * amp * d * np.sin(theta) / k2
    return out
