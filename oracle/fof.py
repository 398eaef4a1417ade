"""Oracle: friends-of-friends (FoF) halo finding on the particles' fixed-point coordinates.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passage: §2.3 (the N-body shop FoF finder run on the fly, 19% of the run time in Table 1)
and §3.2 (haloes identified with linking length 0.2 times the mean particle separation; 0.37 for
2LPT).  Two particles are friends when their periodic distance is at most the linking length;
a group is a connected component of the friendship graph (friends of friends).

Readings where the paper is silent: the distance is measured exactly on the fixed-point coordinates
G of the deposit (20 fractional bits per mesh cell), with the linking length
l = rint(b * (N / N_p) * 2^20) in the same units and the test d^2 <= l^2 in integers, so no
rounding decides a link.  A group is labelled by its smallest particle id.  A halo is a group of at
least n_min members; its position is the periodic centre of mass, computed as
G_root + (sum of minimum-image offsets G_j - G_root) / size in FP64 from exact integer sums, then
wrapped into [0, N) mesh cells.  Haloes are listed in increasing label order.

Library primitives serve as steps: scipy's connected components, and for large inputs scipy's
periodic k-d tree as a candidate pair search (radius slightly above l, then the exact integer test
decides), which ``tests/test_oracle_fof.py`` pins against the brute-force search over all pairs.
"""

from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree
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


def friend_pairs_kdtree(g, nmesh: int, ell: int):
    """The pairs of ``friend_pairs`` from a periodic k-d tree: candidates within l (1 + 1e-9)
    (G / 2^20 is exact in FP64), then the exact integer test."""
    modulus = nmesh << cic.FRAC_BITS
    x = g.T.astype(np.float64) / float(1 << cic.FRAC_BITS)
    tree = cKDTree(x, boxsize=float(nmesh))
    pairs = tree.query_pairs(ell / float(1 << cic.FRAC_BITS) * (1.0 + 1e-9), output_type="ndarray")
    if pairs.size == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    i = np.minimum(pairs[:, 0], pairs[:, 1]).astype(np.int64)
    j = np.maximum(pairs[:, 0], pairs[:, 1]).astype(np.int64)
    d = _wrap(g[:, j] - g[:, i], modulus)
    keep = np.all(np.abs(d) <= ell, axis=0) & (np.sum(d * d, axis=0) <= ell * ell)
    return i[keep], j[keep]


def fof(s, np_side: int, nmesh: int, b: float = 0.2, n_min: int = 1, search: str = "auto"):
    """FoF groups of the particles at displacement s [3, n] (float32 mesh cells).

    Returns dict(label [n] (smallest id in the group), size [n] (members of the particle's group),
    halo_label, halo_size [h], halo_pos [3, h] (mesh cells, FP64)) for groups of >= n_min members.
    """
    g = cic.fixed_point_coords(s, np_side, nmesh)
    n = g.shape[1]
    modulus = nmesh << cic.FRAC_BITS
    ell = linking_length_fixed(b, np_side, nmesh)
    use_tree = search == "kdtree" or (search == "auto" and n > 20000)
    i, j = friend_pairs_kdtree(g, nmesh, ell) if use_tree else friend_pairs(g, nmesh, ell)
    graph = coo_matrix((np.ones(i.size), (i, j)), shape=(n, n))
    _, comp = connected_components(graph, directed=False)
    root = np.full(comp.max() + 1, n, dtype=np.int64)
    np.minimum.at(root, comp, np.arange(n))
    label = root[comp]
    counts = np.bincount(label, minlength=n)
    size = counts[label]
    roots = np.nonzero((label == np.arange(n)) & (counts >= n_min))[0]
    # exact int64 sums of the minimum-image offsets of every member to its root
    off = _wrap(g - g[:, label], modulus)
    tot = np.zeros((3, n), dtype=np.int64)
    for a in range(3):
        np.add.at(tot[a], label, off[a])
    com = g[:, roots].astype(np.float64) + tot[:, roots].astype(np.float64) / counts[roots].astype(np.float64)
    pos = np.mod(com, float(modulus)) / float(1 << cic.FRAC_BITS)
    return dict(label=label, size=size, halo_label=roots, halo_size=counts[roots], halo_pos=pos)
