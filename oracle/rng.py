"""Oracle: the seeded Gaussian white noise of the initial conditions.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passage: the initial conditions are 2LPT displacements of Gaussian random modes drawn by a
2LPTic-style code from a random seed (§2.3).  The paper does not name its generator; this oracle
fixes one (a reading): the real-space white noise on the N_p^3 Lagrangian lattice is drawn from the
counter-based generator Philox-4x32-10 (Salmon, Moraes, Dror & Shaw 2011, "Parallel random numbers:
as easy as 1, 2, 3"), keyed by the seed, then made Gaussian by the Box-Muller transform.

  * Philox-4x32-10: a counter of four 32-bit words and a key of two.  Ten rounds; each round takes
    the 64-bit products M0 c0 and M1 c2 (M0 = 0xD2511F53, M1 = 0xCD9E8D57) and returns
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); between rounds the key
    advances by the Weyl constants (0x9E3779B9, 0xBB67AE85) modulo 2^32.
  * Lattice site i (the particle id (ix N_p + iy) N_p + iz) takes counter j = floor(i / 4) =
    (j mod 2^32, j div 2^32, 0, 0) and key (seed mod 2^32, seed div 2^32).  The output words
    (x0, x1) serve sites 4j and 4j+1, (x2, x3) sites 4j+2 and 4j+3.
  * Box-Muller on a word pair (a, b): u1 = ((a >> 8) + 1) 2^-24 in (0, 1], u2 = (b >> 8) 2^-24 in
    [0, 1), r = sqrt(-2 ln u1); the first site gets r cos(2 pi u2), the second r sin(2 pi u2).

The 32-bit words are exact integers; the Gaussians here are FP64 (the GPU evaluates the same
formula in FP32, so the two agree to FP32 rounding, and their words bit for bit).
"""

from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32(ctr, key, rounds: int = 10):
    """Philox-4x32 with `rounds` rounds of counters ctr [4, m] under keys key [2, m] (or [2]);
    returns the output words [4, m] as uint64 arrays holding 32-bit values."""
    c = [np.asarray(w, dtype=np.uint64) & MASK for w in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & MASK
    k1 = np.asarray(key[1], dtype=np.uint64) & MASK
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = np.uint64(M0) * c[0]            # exact: both factors < 2^32
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def lattice_words(seed: int, n_sites: int):
    """The Philox words of the first ceil(n_sites / 4) counters of `seed`: uint64 array [4, m]."""
    m = (n_sites + 3) // 4
    j = np.arange(m, dtype=np.uint64)
    ctr = [j & np.uint64(MASK), j >> np.uint64(32), np.zeros(m, np.uint64), np.zeros(m, np.uint64)]
    return np.stack(philox4x32(ctr, (seed & MASK, (seed >> 32) & MASK)))


def box_muller(a, b):
    """The Gaussian pair of a word pair (module docstring), FP64."""
    u1 = ((np.asarray(a, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (np.asarray(b, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def white_noise(seed: int, np_side: int):
    """Unit Gaussian white noise of `seed` on the np_side^3 lattice, float64 [np_side^3] in particle-id
    order (§2.3 initial conditions)."""
    n = np_side ** 3
    x = lattice_words(seed, n)
    g0, g1 = box_muller(x[0], x[1])
    g2, g3 = box_muller(x[2], x[3])
    out = np.stack([g0, g1, g2, g3], axis=1).reshape(-1)
    return out[:n]
