"""Oracle: cloud-in-cell (CIC) mass assignment and interpolation on the periodic PM mesh.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages: the PM force assigns particles to a uniform mesh and interpolates the force
back (§2.3, the (3 x 1296)^3 PM mesh; Appendix A, the PM force resolution) and the power
spectrum assigns densities with CIC (§3.3).  The paper does not define the arithmetic of the
assignment; this oracle fixes it as a deterministic fixed-point scheme (a reading, not the paper's):

  * a particle with lattice index q (per axis, 0..Np-1) and displacement s (PM cells) sits at
    mesh coordinate q*r + s, r = N/Np;
  * its fixed-point coordinate is G = (q*R + rint(s * 2^20)) mod (N * 2^20), R = r * 2^20 an
    integer, rint rounding half to even;
  * cell c = G >> 20, 14-bit fraction f = (G >> 6) & (2^14 - 1);
  * weights along the axis are (2^14 - f) at c and f at c+1; the 8 products (<= 2^42) are added
    to an unsigned 64-bit mesh, so every particle deposits exactly 2^42;
  * density contrast delta = rho * N^3 / (n * 2^42) - 1 (n particles).

The textbook FP64 CIC (``cic_exact_mesh``) is kept beside it for the pins and for stating the
quantisation error of the fixed-point weights.
"""

from __future__ import annotations

import numpy as np

FRAC_BITS = 20                  # fractional bits of the fixed-point coordinate
WEIGHT_BITS = 14                # bits of each per-axis weight
WEIGHT_ONE = 1 << WEIGHT_BITS   # 16384
PARTICLE_MASS = 1 << (3 * WEIGHT_BITS)   # 2^42, the fixed-point mass of one particle


def lattice_indices(np_side: int) -> np.ndarray:
    """Per-axis lattice index [3, n] of particle id = (ix * Np + iy) * Np + iz."""
    ix, iy, iz = np.meshgrid(np.arange(np_side), np.arange(np_side), np.arange(np_side),
                             indexing="ij")
    return np.stack([ix.ravel(), iy.ravel(), iz.ravel()]).astype(np.int64)


def fixed_point_coords(s, np_side: int, nmesh: int) -> np.ndarray:
    """Fixed-point mesh coordinate G [3, n] (int64) of displacement s [3, n] in mesh cells."""
    if (nmesh << FRAC_BITS) % np_side:
        raise ValueError("nmesh * 2^20 must be a multiple of np_side")
    r_fixed = (nmesh << FRAC_BITS) // np_side
    q = lattice_indices(np_side)
    s64 = np.asarray(s, dtype=np.float64)
    g = q * r_fixed + np.rint(s64 * float(1 << FRAC_BITS)).astype(np.int64)
    return np.mod(g, nmesh << FRAC_BITS)


def cells_and_fractions(s, np_side: int, nmesh: int):
    """(cell [3, n] int64, f [3, n] int64) of the fixed-point scheme."""
    g = fixed_point_coords(s, np_side, nmesh)
    return g >> FRAC_BITS, (g >> (FRAC_BITS - WEIGHT_BITS)) & (WEIGHT_ONE - 1)


def cic_fixed_mesh(s, np_side: int, nmesh: int) -> np.ndarray:
    """Unsigned 64-bit fixed-point CIC mesh [N, N, N] of the particles (exact integer sums)."""
    cell, f = cells_and_fractions(s, np_side, nmesh)
    n3 = nmesh
    mesh = np.zeros(n3 ** 3, dtype=np.uint64)
    for dx in (0, 1):
        wx = f[0] if dx else WEIGHT_ONE - f[0]
        ix = (cell[0] + dx) % n3
        for dy in (0, 1):
            wy = f[1] if dy else WEIGHT_ONE - f[1]
            iy = (cell[1] + dy) % n3
            for dz in (0, 1):
                wz = f[2] if dz else WEIGHT_ONE - f[2]
                iz = (cell[2] + dz) % n3
                np.add.at(mesh, (ix * n3 + iy) * n3 + iz, (wx * wy * wz).astype(np.uint64))
    return mesh.reshape(n3, n3, n3)


def delta_from_fixed(mesh: np.ndarray, n_particles: int) -> np.ndarray:
    """Density contrast delta = rho N^3 / (n 2^42) - 1 in FP64."""
    n3 = mesh.size
    return mesh.astype(np.float64) * (n3 / (n_particles * float(PARTICLE_MASS))) - 1.0


def interp_weights_fixed(s, np_side: int, nmesh: int):
    """(cell [3, n], w1 [3, n]) for interpolation: w1 = f / 2^14 is the weight of cell c+1."""
    cell, f = cells_and_fractions(s, np_side, nmesh)
    return cell, f.astype(np.float64) / WEIGHT_ONE


def cic_interp(fields, cell, w1) -> np.ndarray:
    """CIC interpolation of fields [m, N, N, N] at particles (cell, w1): returns [m, n] in FP64."""
    fields = np.asarray(fields, dtype=np.float64)
    n3 = fields.shape[-1]
    out = np.zeros((fields.shape[0], cell.shape[1]), dtype=np.float64)
    for dx in (0, 1):
        wx = w1[0] if dx else 1.0 - w1[0]
        ix = (cell[0] + dx) % n3
        for dy in (0, 1):
            wy = w1[1] if dy else 1.0 - w1[1]
            iy = (cell[1] + dy) % n3
            for dz in (0, 1):
                wz = w1[2] if dz else 1.0 - w1[2]
                iz = (cell[2] + dz) % n3
                out += fields[:, ix, iy, iz] * (wx * wy * wz)
    return out


def cic_exact_mesh(x, nmesh: int) -> np.ndarray:
    """Textbook FP64 CIC: particle count per cell for positions x [3, n] in mesh cells."""
    x = np.mod(np.asarray(x, dtype=np.float64), nmesh)
    c = np.floor(x).astype(np.int64)
    t = x - c
    mesh = np.zeros(nmesh ** 3, dtype=np.float64)
    for dx in (0, 1):
        wx = t[0] if dx else 1.0 - t[0]
        for dy in (0, 1):
            wy = t[1] if dy else 1.0 - t[1]
            for dz in (0, 1):
                wz = t[2] if dz else 1.0 - t[2]
                idx = (((c[0] + dx) % nmesh) * nmesh + (c[1] + dy) % nmesh) * nmesh \
                    + (c[2] + dz) % nmesh
                np.add.at(mesh, idx, wx * wy * wz)
    return mesh.reshape(nmesh, nmesh, nmesh)
