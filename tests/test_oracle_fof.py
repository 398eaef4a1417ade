"""Pins of the oracle's friends-of-friends finder (§2.3, §3.2: linking length 0.2 times the mean
particle separation): closed-form lattices, chains, periodic wrap-around, the exact boundary of the
link test, the periodic centre of mass, and an independent breadth-first search on FP64
distances."""

import collections

import numpy as np
import pytest

from oracle import cic, fof

NP, NM = 6, 12          # mean particle separation 2 mesh cells


def _groups(label):
    out = collections.defaultdict(set)
    for i, l in enumerate(label):
        out[int(l)].add(i)
    return sorted(tuple(sorted(v)) for v in out.values())


@pytest.mark.parametrize("b,ngroups", [(0.2, NP ** 3), (0.99, NP ** 3), (1.0, 1), (1.2, 1)])
def test_unperturbed_lattice(b, ngroups):
    """Nearest neighbours sit exactly one mean separation apart: b < 1 leaves singletons, b = 1
    (distance equal to the linking length, which links) joins the whole periodic lattice."""
    r = fof.fof(np.zeros((3, NP ** 3), dtype=np.float32), NP, NM, b)
    assert len(set(r["label"].tolist())) == ngroups
    if ngroups == 1:
        assert np.all(r["label"] == 0) and np.all(r["size"] == NP ** 3)


def _far_apart():
    """Displacements that park particle i at a distinct, well separated point of the box."""
    n = NP ** 3
    q = cic.lattice_indices(NP).astype(np.float64) * (NM / NP)
    return q, np.zeros((3, n))


def _place(points):
    """s such that particle i (i < len(points)) sits at points[i]; the rest stay on the lattice
    (2 cells apart, not linked at b = 0.2)."""
    q, s = _far_apart()
    for i, p in enumerate(points):
        s[:, i] = np.asarray(p, dtype=np.float64) - q[:, i]
    return s.astype(np.float32)


def test_chain_links_friends_of_friends():
    """Four particles 0.375 cells apart along x (l = 0.4 cells at b = 0.2): each only touches its
    neighbours, yet all four form one group; at 0.4375 cells apart none link."""
    ell = 0.2 * NM / NP
    pts = [(5.0 + 0.375 * k, 5.25, 5.25) for k in range(4)]
    r = fof.fof(_place(pts), NP, NM, 0.2)
    assert set(r["label"][:4].tolist()) == {0} and r["size"][0] == 4
    assert 0.375 * 2 > ell   # the ends are not direct friends
    pts = [(5.0 + 0.4375 * k, 5.25, 5.25) for k in range(4)]
    r = fof.fof(_place(pts), NP, NM, 0.2)
    assert r["label"][:4].tolist() == [0, 1, 2, 3]


def test_links_across_the_periodic_boundary_and_centre_of_mass():
    """Two particles 0.125 cells either side of x = 0 link through the boundary; their centre of
    mass is x = 0 (wrapped into [0, N))."""
    pts = [(0.125, 3.25, 7.25), (NM - 0.125, 3.25, 7.25)]
    r = fof.fof(_place(pts), NP, NM, 0.2, n_min=2)
    assert r["label"][0] == 0 and r["label"][1] == 0
    assert r["halo_label"].tolist() == [0] and r["halo_size"].tolist() == [2]
    np.testing.assert_allclose(r["halo_pos"][:, 0], [0.0, 3.25, 7.25], atol=0)


def test_link_test_is_exact_at_the_linking_length():
    """Fixed-point separation exactly l links, l + 2^-20 cells does not."""
    ell = fof.linking_length_fixed(0.2, NP, NM) / float(1 << 20)
    for gap, linked in ((ell, True), (ell + 2.0 ** -20, False)):
        r = fof.fof(_place([(4.0, 4.0, 4.0), (4.0 + gap, 4.0, 4.0)]), NP, NM, 0.2)
        assert (r["label"][1] == 0) == linked


def test_halo_threshold_and_order():
    # odd coordinates keep both chains more than l away from the particles left on the lattice
    pts = [(1.0 + 0.3 * k, 1.0, 1.0) for k in range(3)] + [(7.0, 7.0 + 0.3 * k, 7.0) for k in range(5)]
    r = fof.fof(_place(pts), NP, NM, 0.2, n_min=4)
    assert r["halo_label"].tolist() == [3] and r["halo_size"].tolist() == [5]
    np.testing.assert_allclose(r["halo_pos"][:, 0], [7.0, 7.6, 7.0], rtol=0, atol=1e-6)
    r = fof.fof(_place(pts), NP, NM, 0.2, n_min=3)
    assert r["halo_label"].tolist() == [0, 3]


def test_matches_breadth_first_search_on_float_distances():
    """Clustered random particles: groups equal a plain BFS on FP64 periodic distances (the
    configuration has no pair within 1e-6 cells of the linking length, so both tests agree)."""
    rng = np.random.default_rng(3)
    npd, nm = 8, 16
    n = npd ** 3
    q = cic.lattice_indices(npd).astype(np.float64) * (nm / npd)
    centres = rng.uniform(0, nm, size=(3, 12))
    pick = rng.integers(0, 12, size=n)
    x = centres[:, pick] + rng.normal(0, 0.35, size=(3, n))
    s = (x - q).astype(np.float32)
    r = fof.fof(s, npd, nm, 0.2)
    g = cic.fixed_point_coords(s, npd, nm).astype(np.float64) / float(1 << 20)
    ell = fof.linking_length_fixed(0.2, npd, nm) / float(1 << 20)
    d = g[:, :, None] - g[:, None, :]
    d = d - nm * np.rint(d / nm)
    dist = np.sqrt(np.sum(d * d, axis=0))
    assert np.min(np.abs(dist - ell)) > 1e-6
    adj = dist <= ell
    label = -np.ones(n, dtype=np.int64)
    for start in range(n):
        if label[start] >= 0:
            continue
        label[start] = start
        queue = collections.deque([start])
        while queue:
            a = queue.popleft()
            for b_ in np.nonzero(adj[a] & (label < 0))[0]:
                label[b_] = start
                queue.append(b_)
    assert _groups(r["label"]) == _groups(label)
    assert np.array_equal(r["label"], label)        # BFS from increasing starts labels by min id
    assert len(set(label.tolist())) < n // 4        # the configuration is really clustered


@pytest.mark.parametrize("b", [0.2, 0.37, 0.6])
def test_kdtree_candidates_equal_brute_force(b):
    """The k-d tree search used for large inputs finds exactly the brute-force friend pairs."""
    rng = np.random.default_rng(int(b * 100))
    npd, nm = 10, 20
    q = cic.lattice_indices(npd).astype(np.float64) * (nm / npd)
    centres = rng.uniform(0, nm, size=(3, 30))
    x = centres[:, rng.integers(0, 30, size=npd ** 3)] + rng.normal(0, 0.5, size=(3, npd ** 3))
    s = (x - q).astype(np.float32)
    g = cic.fixed_point_coords(s, npd, nm)
    ell = fof.linking_length_fixed(b, npd, nm)
    i1, j1 = fof.friend_pairs(g, nm, ell)
    i2, j2 = fof.friend_pairs_kdtree(g, nm, ell)
    assert i1.size > 100
    assert sorted(zip(i1.tolist(), j1.tolist())) == sorted(zip(i2.tolist(), j2.tolist()))
    a = fof.fof(s, npd, nm, b, n_min=3, search="brute")
    k = fof.fof(s, npd, nm, b, n_min=3, search="kdtree")
    for key in ("label", "size", "halo_label", "halo_size", "halo_pos"):
        assert np.array_equal(a[key], k[key]), key
