"""Oracle: matter power spectrum estimator.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passage: §3.3 (matter power spectrum).  CIC density on a mesh, FFT, keep the modes
{k_z > 0} U {k_z = 0, k_y > 0} U {k_z = 0, k_y = 0, k_x > 0} of the k_z >= 0 half so that no
mode is counted twice, P(k) = V^-1 <|delta(k)|^2> per bin, plotted against the mean |k| of the
bin's modes.  The paper corrects the CIC smoothing and aliasing with the procedure of Jing
(2005); ``power_spectrum(..., cic_correct=True, n_particles=n)`` applies that correction for a
locally flat spectrum: per mode P = P_raw / C2(k) - V/n, with the alias-summed CIC window
C2(k) = sum_n W^2(k + 2 k_N n) = prod_i (1 - (2/3) sin^2(pi m_i / N)) (the flat-spectrum form of
Jing's correction; his iteration on a local power-law slope is not applied).

Readings where the paper is silent: delta(k) = (V/N^3) sum_x delta_x e^{-i k.x}, so P = V |DFT|^2 / N^6.  Bins
are log spaced between the fundamental k_f = 2 pi / L and the Nyquist k_N = pi N / L (the paper
uses linear bins of 0.01 h/Mpc; the 64 log bins are the workload's).  A mode's bin is decided on
its integer |m|^2 against integer edges T_b = ceil(e_b^2 - 1e-9), e_b = (N/2)^(b/nbins), so no
floating-point rounding can move a mode between bins.  No smoothing/alias correction and no shot
noise subtraction.
"""

from __future__ import annotations

import math

import numpy as np

from . import fourier


def bin_edges_m2(nmesh: int, nbins: int) -> np.ndarray:
    """Integer lower edges T_0..T_nbins of the bins in |m|^2 (T_nbins = (N/2)^2, exclusive)."""
    half = nmesh / 2.0
    e2 = [half ** (2.0 * b / nbins) for b in range(nbins + 1)]
    return np.array([math.ceil(v - 1e-9) for v in e2], dtype=np.int64)


def half_space_mask(nmesh: int) -> np.ndarray:
    """Boolean mask on the half spectrum [N, N, N/2+1] of the independent modes of §3.3."""
    mx, my, mz = fourier.mode_grids(nmesh)
    return (mz > 0) | ((mz == 0) & (my > 0)) | ((mz == 0) & (my == 0) & (mx > 0))


def cic_alias_sum(mx, my, mz, n: int):
    """C2(m) = prod_i (1 - (2/3) sin^2(pi m_i / N)): the CIC window squared summed over aliases."""
    out = 1.0
    for m in (mx, my, mz):
        out = out * (1.0 - (2.0 / 3.0) * np.sin(np.pi * np.asarray(m, dtype=np.float64) / n) ** 2)
    return out


def power_spectrum(delta: np.ndarray, box: float, nbins: int, cic_correct: bool = False,
                   n_particles: int | None = None):
    """(k_mean [nbins], P [nbins], n_modes [nbins]) of a density contrast field delta [N, N, N]."""
    n = delta.shape[0]
    dk = fourier.rfft3(delta)
    pmode = np.abs(dk) ** 2 * (box ** 3 / float(n) ** 6)
    mx, my, mz = fourier.mode_grids(n)
    if cic_correct:
        pmode = pmode / cic_alias_sum(mx, my, mz, n) - box ** 3 / float(n_particles)
    m2 = mx * mx + my * my + mz * mz
    m2 = np.broadcast_to(m2, dk.shape)
    kmag = np.sqrt(m2.astype(np.float64)) * (2.0 * np.pi / box)
    mask = half_space_mask(n)
    edges = bin_edges_m2(n, nbins)
    b = np.searchsorted(edges, m2, side="right") - 1          # T_b <= m2 < T_{b+1}
    keep = mask & (b >= 0) & (b < nbins)
    bsel = b[keep]
    counts = np.bincount(bsel, minlength=nbins)[:nbins]
    psum = np.bincount(bsel, weights=pmode[keep], minlength=nbins)[:nbins]
    ksum = np.bincount(bsel, weights=kmag[keep], minlength=nbins)[:nbins]
    with np.errstate(divide="ignore", invalid="ignore"):
        kmean = np.where(counts > 0, ksum / np.maximum(counts, 1), 0.0)
        pk = np.where(counts > 0, psum / np.maximum(counts, 1), 0.0)
    return kmean, pk, counts.astype(np.int64)
