"""Oracle: friends-of-friends (FoF) halo finding on the particles' fixed-point coordinates.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passage: §2.3 (the N-body shop FoF finder run on the fly, 19% of the run time in Table 1)
and §3.2 (haloes identified with linking length 0.2 times the mean particle separation; 0.37 for
2LPT).  Two particles are friends when their periodic distance is at most the linking length;
a group is a connected component of the friendship graph (friends of friends).

Readings (reading 20): the distance is measured exactly on the fixed-point coordinates
G of the deposit (20 fractional bits per mesh cell), with the linking length
l = rint(b * (N / N_p) * 2^20) in the same units and the test d^2 <= l^2 in integers, so no
rounding decides a link.  A group is labelled by its smallest particle id.  A halo is a group of at
least n_min members; its position is the periodic centre of mass, computed as
G_root + (sum of minimum-image offsets G_j - G_root) / size in FP64 from exact integer sums, then
wrapped into [0, N) mesh cells.  Haloes are listed in increasing label order.

A library primitive (scipy's connected components) serves as the component step; the pair search
is brute force over all pairs.
"""

from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from . import cic


def linking_length_fixed(b: float, np_side: int, nmesh: int) -> int:
    """l = rint(b * (N / N_p) * 2^20), round half to even."""
    return int(np.rint(b * (nmesh / np_side) * float(1 << cic.FRAC_BITS)))


def _wrap(d, modulus: int):
    """Minimum image of integer differences d in (-modulus, modulus)."""
    d = np.where(d > modulus // 2, d - modulus, d)
    return np.where(d < -(modulus // 2), d + modulus, d)


def friend_pairs(g, nmesh: int, ell: int):
    """All pairs (i < j) with periodic integer distance^2 <= ell^2 (brute force, O(n^2))."""
    modulus = nmesh << cic.FRAC_BITS
    n = g.shape[1]
    ii, jj = [], []
    for i in range(n - 1):
        d = _wrap(g[:, i + 1:] - g[:, i:i + 1], modulus)
        near = np.all(np.abs(d) <= ell, axis=0)
        idx = np.nonzero(near)[0]
        if idx.size:
            dd = d[:, idx]
            d2 = np.sum(dd * dd, axis=0)
            sel = idx[d2 <= ell * ell]
            ii.append(np.full(sel.size, i, dtype=np.int64))
            jj.append(sel + i + 1)
    if not ii:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    return np.concatenate(ii), np.concatenate(jj)


def fof(s, np_side: int, nmesh: int, b: float = 0.2, n_min: int = 1):
    """FoF groups of the particles at displacement s [3, n] (float32 mesh cells).

    Returns dict(label [n] (smallest id in the group), size [n] (members of the particle's group),
    halo_label, halo_size [h], halo_pos [3, h] (mesh cells, FP64)) for groups of >= n_min members.
    """
    g = cic.fixed_point_coords(s, np_side, nmesh)
    n = g.shape[1]
    modulus = nmesh << cic.FRAC_BITS
    ell = linking_length_fixed(b, np_side, nmesh)
    i, j = friend_pairs(g, nmesh, ell)
    graph = coo_matrix((np.ones(i.size), (i, j)), shape=(n, n))
    _, comp = connected_components(graph, directed=False)
    root = np.full(comp.max() + 1, n, dtype=np.int64)
    np.minimum.at(root, comp, np.arange(n))
    label = root[comp]
    counts = np.bincount(label, minlength=n)
    size = counts[label]
    roots = np.nonzero((label == np.arange(n)) & (counts >= n_min))[0]
    pos = np.zeros((3, roots.size))
    for h, r in enumerate(roots):
        members = np.nonzero(label == r)[0]
        off = _wrap(g[:, members] - g[:, r:r + 1], modulus)
        tot = off.sum(axis=1)                                   # exact int64 sums
        com = g[:, r].astype(np.float64) + tot.astype(np.float64) / float(members.size)
        com = np.mod(com, float(modulus))
        pos[:, h] = com / float(1 << cic.FRAC_BITS)
    return dict(label=label, size=size, halo_label=roots, halo_size=counts[roots], halo_pos=pos)
