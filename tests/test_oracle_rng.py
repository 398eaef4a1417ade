"""Pins of the oracle's seeded white noise (§2.3 Gaussian modes from a seed; the generator is a
reading: Philox-4x32-10 and Box-Muller): the published known-answer vectors of the generator
(tests/golden/philox4x32_10_kat.txt, with its citation), the uniform maps' end points, the Box-Muller
radius identity and the Gaussian moments."""

import math
import os

import numpy as np
import pytest

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answer_vectors():
    rows = kat_rows()
    assert len(rows) == 3
    for w in rows:
        out = rng.philox4x32([[w[0]], [w[1]], [w[2]], [w[3]]], (w[4], w[5]))
        assert [int(o[0]) for o in out] == w[6:]


def test_philox_vectorised_counters_match_one_by_one():
    # the lattice counters (j, 0, 0, 0) evaluated together equal single evaluations
    seed = 0x1234_5678_9ABC
    x = rng.lattice_words(seed, 4 * 37)
    for j in (0, 1, 17, 36):
        one = rng.philox4x32([[j], [0], [0], [0]], (seed & 0xFFFFFFFF, seed >> 32))
        assert [int(o[0]) for o in one] == [int(x[q, j]) for q in range(4)]


def test_uniform_end_points():
    # u1 = ((a >> 8) + 1) 2^-24 lies in (0, 1]; u2 = (b >> 8) 2^-24 in [0, 1)
    z0, z1 = rng.box_muller(np.array([0xFFFFFFFF]), np.array([0]))
    assert z0[0] == 0.0 and z1[0] == 0.0                       # u1 = 1: r = 0
    z0, z1 = rng.box_muller(np.array([0]), np.array([0]))
    r = math.sqrt(-2.0 * math.log(2.0 ** -24))                   # the largest radius, 5.77
    assert z0[0] == pytest.approx(r, rel=1e-15) and z1[0] == 0.0
    z0, z1 = rng.box_muller(np.array([0]), np.array([0x40000000]))   # u2 = 1/4: the sine branch
    assert abs(z0[0]) < 1e-15 and z1[0] == pytest.approx(r, rel=1e-15)


def test_box_muller_pairs_share_their_radius():
    seed, npd = 7, 16
    x = rng.lattice_words(seed, npd ** 3)
    wn = rng.white_noise(seed, npd)
    u1 = ((x[0] >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    np.testing.assert_allclose(wn[0::4] ** 2 + wn[1::4] ** 2, -2.0 * np.log(u1), rtol=1e-12, atol=1e-300)
    u1b = ((x[2] >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    np.testing.assert_allclose(wn[2::4] ** 2 + wn[3::4] ** 2, -2.0 * np.log(u1b), rtol=1e-12, atol=1e-300)


def test_white_noise_moments_and_independence():
    npd = 96   # 884,736 sites
    a = rng.white_noise(11, npd)
    b = rng.white_noise(12, npd)
    n = a.size
    assert abs(a.mean()) < 5.0 / math.sqrt(n)
    assert abs(a.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    kurt = np.mean(a ** 4) / np.mean(a ** 2) ** 2
    assert abs(kurt - 3.0) < 5.0 * math.sqrt(24.0 / n)
    assert abs(np.mean(a ** 3)) < 5.0 * math.sqrt(15.0 / n)
    # tails: P(|z| > 3) = 0.0026998
    frac = np.mean(np.abs(a) > 3.0)
    assert abs(frac - 0.0026998) < 5.0 * math.sqrt(0.0027 / n)
    # different seeds and neighbouring sites are uncorrelated
    assert abs(np.mean(a * b)) < 5.0 / math.sqrt(n)
    assert abs(np.mean(a[:-1] * a[1:])) < 5.0 / math.sqrt(n)
    assert abs(np.mean(a[0::4] * a[1::4])) < 5.0 / math.sqrt(n / 4)   # the cos/sin pair of one radius
