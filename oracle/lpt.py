"""Oracle: Gaussian initial field and 2LPT displacements Psi1, Psi2.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages: the 2LPT growing mode x = q + D1 Psi1 + D2 Psi2 (§2.1) generated by a 2LPTic
style code from Gaussian random modes (§2.3).  The paper does not write the 2LPT field equations;
the textbook ones are used (a reading; signs fixed by D2 < 0):

    Psi1 = -grad phi1,  nabla^2 phi1 = delta_L;           Psi1(k) =  i k delta_L / k^2
    phi1_ij(k) = k_i k_j delta_L / k^2
    S = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2)
    Psi2 = +grad phi2,  nabla^2 phi2 = S;                 Psi2(k) = -i k S(k) / k^2

delta_L is the linear density at a = 1 on the particle lattice: W = rfft(w) of the white noise
w ~ N(0, 1) (one value per lattice site, an input), delta_L(k) = W sqrt(P(k) / V_cell) with
V_cell = (L / Np)^3 and delta_L(0) = 0.  k in h/Mpc is 2 pi m / L.  A single factor k_j is 0 on its
Nyquist plane; the diagonal k_i k_i keeps its Nyquist value (reading 6).
"""

from __future__ import annotations

import numpy as np

from . import cosmology, fourier


def linear_density_k(white_noise: np.ndarray, p: cosmology.Params) -> np.ndarray:
    """delta_L(k) on the half spectrum of the Np^3 lattice."""
    npd = p.np_side
    w = np.asarray(white_noise, dtype=np.float64).reshape(npd, npd, npd)
    wk = fourier.rfft3(w)
    mx, my, mz = fourier.mode_grids(npd)
    kf = 2.0 * np.pi / p.box
    kmag = np.sqrt((mx * mx + my * my + mz * mz).astype(np.float64)) * kf
    vcell = (p.box / npd) ** 3
    amp = cosmology.power_amplitude(p)
    pk = np.where(kmag > 0, cosmology.linear_power(np.where(kmag > 0, kmag, 1.0), p, amp), 0.0)
    return wk * np.sqrt(pk / vcell)


def _wavenumbers(npd: int, box: float):
    mx, my, mz = fourier.mode_grids(npd)
    kf = 2.0 * np.pi / box
    mm = (mx, my, mz)
    k_full = [m.astype(np.float64) * kf for m in mm]
    k_odd = [fourier.odd_mode(m, npd).astype(np.float64) * kf for m in mm]
    k2 = k_full[0] ** 2 + k_full[1] ** 2 + k_full[2] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_k2 = np.where(k2 > 0, 1.0 / k2, 0.0)
    return k_full, k_odd, inv_k2


def first_order(dk: np.ndarray, npd: int, box: float) -> np.ndarray:
    """Psi1 [3, Np, Np, Np] in Mpc/h from delta_L(k): Psi1(k) = i k delta_L / k^2."""
    _, k_odd, inv_k2 = _wavenumbers(npd, box)
    return np.stack([fourier.irfft3(1j * k_odd[j] * dk * inv_k2, npd) for j in range(3)])


def second_order_source(dk: np.ndarray, npd: int, box: float) -> np.ndarray:
    """S = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2) in real space, phi1_ij(k) = k_i k_j delta_L / k^2."""
    k_full, k_odd, inv_k2 = _wavenumbers(npd, box)

    def hess(i, j):
        kk = k_full[i] * k_full[i] if i == j else k_odd[i] * k_odd[j]
        return fourier.irfft3(kk * dk * inv_k2, npd)

    p00, p11, p22 = hess(0, 0), hess(1, 1), hess(2, 2)
    p01, p02, p12 = hess(0, 1), hess(0, 2), hess(1, 2)
    return p00 * p11 + p00 * p22 + p11 * p22 - p01 ** 2 - p02 ** 2 - p12 ** 2


def second_order(dk: np.ndarray, npd: int, box: float) -> np.ndarray:
    """Psi2 [3, Np, Np, Np] in Mpc/h: Psi2(k) = -i k S(k) / k^2."""
    _, k_odd, inv_k2 = _wavenumbers(npd, box)
    sk = fourier.rfft3(second_order_source(dk, npd, box))
    return np.stack([fourier.irfft3(-1j * k_odd[j] * sk * inv_k2, npd) for j in range(3)])


def displacements(white_noise: np.ndarray, p: cosmology.Params):
    """(Psi1, Psi2) as [3, n] arrays in PM mesh cells (L / N) for particle id (ix*Np+iy)*Np+iz."""
    dk = linear_density_k(white_noise, p)
    to_cells = p.nmesh / p.box
    psi1 = first_order(dk, p.np_side, p.box)
    psi2 = second_order(dk, p.np_side, p.box)
    return psi1.reshape(3, -1) * to_cells, psi2.reshape(3, -1) * to_cells
