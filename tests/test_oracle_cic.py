"""Pins of the oracle's CIC assignment and interpolation (§2.3 PM mesh, §3.3 CIC) against the
textbook cloud-overlap definition (brute force), exact invariants and the fixed-point reading."""

import itertools

import numpy as np
import pytest

import cola_inputs
from oracle import cic


def brute_force_cic(x, nmesh):
    """Cloud-overlap definition: weight of cell c = prod_a max(0, 1 - |x_a - c_a|) (periodic)."""
    mesh = np.zeros((nmesh,) * 3)
    for p in range(x.shape[1]):
        for c in itertools.product(range(nmesh), repeat=3):
            w = 1.0
            for a in range(3):
                d = abs(x[a, p] - c[a]) % nmesh
                d = min(d, nmesh - d)
                w *= max(0.0, 1.0 - d)
            mesh[c] += w
    return mesh


def test_exact_cic_matches_cloud_overlap_brute_force():
    rng = np.random.default_rng(11)
    x = rng.uniform(-3, 9, size=(3, 7))
    np.testing.assert_allclose(cic.cic_exact_mesh(x, 6), brute_force_cic(x, 6), atol=1e-13)


def test_fixed_equals_exact_on_dyadic_positions():
    # positions on the 2^-14 grid: the 14-bit weights are exact, so mesh / 2^42 == textbook CIC
    npd, nm = 4, 8
    rng = np.random.default_rng(3)
    s = (rng.integers(-5 * 2 ** 14, 5 * 2 ** 14, size=(3, npd ** 3)) / 2.0 ** 14).astype(np.float32)
    fixed = cic.cic_fixed_mesh(s, npd, nm).astype(np.float64) / cic.PARTICLE_MASS
    x = cic.lattice_indices(npd) * (nm // npd) + s.astype(np.float64)
    np.testing.assert_array_equal(fixed, cic.cic_exact_mesh(x, nm))


def test_total_mass_is_exact():
    s = cola_inputs.random_displacements(8, seed=5, amplitude=7.0)
    mesh = cic.cic_fixed_mesh(s, 8, 12)
    assert int(mesh.sum(dtype=np.uint64)) == 8 ** 3 * cic.PARTICLE_MASS


@pytest.mark.parametrize("shift", [0.0, 0.5, -0.5])
def test_uniform_lattice_r1_gives_zero_contrast(shift):
    npd = 8
    s = np.full((3, npd ** 3), shift, dtype=np.float32)
    mesh = cic.cic_fixed_mesh(s, npd, npd)
    assert np.all(mesh == cic.PARTICLE_MASS)
    assert np.all(cic.delta_from_fixed(mesh, npd ** 3) == 0.0)


def test_uniform_lattice_r2_has_only_nyquist_modes():
    npd, nm = 6, 12
    s = np.zeros((3, npd ** 3), dtype=np.float32)
    delta = cic.delta_from_fixed(cic.cic_fixed_mesh(s, npd, nm), npd ** 3)
    dk = np.fft.fftn(delta)
    m = np.fft.fftfreq(nm, 1.0 / nm).round().astype(int)
    nyq = (np.abs(m) == nm // 2)
    on_nyq = nyq[:, None, None] | nyq[None, :, None] | nyq[None, None, :]
    assert np.abs(dk[~on_nyq]).max() < 1e-10


def test_round_half_to_even_and_wrap():
    # s * 2^20 = 0.5 rounds to 0, 1.5 to 2, -0.5 to 0; coordinates wrap mod N * 2^20
    s = np.zeros((3, 8), dtype=np.float32)
    s[0, 0] = np.float32(0.5 / 2 ** 20)
    s[0, 1] = np.float32(1.5 / 2 ** 20)
    s[0, 2] = np.float32(-0.5 / 2 ** 20)
    s[0, 3] = np.float32(-1.25)              # lattice x = 0 -> wraps to N - 1.25
    g = cic.fixed_point_coords(s, 2, 4)
    assert g[0, 0] == 0 and g[0, 1] == 2 and g[0, 2] == 0
    assert g[0, 3] == (4 << 20) - int(1.25 * 2 ** 20)


def test_interpolation_reproduces_trilinear_fields():
    # CIC interpolation is exact for fields linear in each coordinate (away from the wrap)
    nm, npd = 16, 4
    rng = np.random.default_rng(8)
    s = (rng.integers(0, 2 * 2 ** 14, size=(3, npd ** 3)) / 2.0 ** 14).astype(np.float32)
    g = np.meshgrid(*(np.arange(nm, dtype=np.float64),) * 3, indexing="ij")
    field = 0.3 + 1.5 * g[0] - 0.7 * g[1] + 0.25 * g[2] + 0.01 * g[0] * g[1] * g[2]
    cell, w1 = cic.interp_weights_fixed(s, npd, nm)
    val = cic.cic_interp(field[None], cell, w1)[0]
    x = cic.lattice_indices(npd) * (nm // npd) + s.astype(np.float64)
    expect = 0.3 + 1.5 * x[0] - 0.7 * x[1] + 0.25 * x[2] + 0.01 * x[0] * x[1] * x[2]
    np.testing.assert_allclose(val, expect, rtol=0, atol=1e-12)


def test_deposit_and_interpolation_are_transposes():
    # sum_c rho_c f_c == 2^42 sum_p interp(f)(x_p): same cells and weights on both sides
    npd, nm = 6, 12
    s = cola_inputs.random_displacements(npd, seed=2, amplitude=4.0)
    f = cola_inputs.random_field((nm, nm, nm), seed=9).astype(np.float64)
    rho = cic.cic_fixed_mesh(s, npd, nm).astype(np.float64)
    cell, w1 = cic.interp_weights_fixed(s, npd, nm)
    lhs = float((rho * f).sum())
    rhs = float(cic.cic_interp(f[None], cell, w1)[0].sum()) * cic.PARTICLE_MASS
    assert lhs == pytest.approx(rhs, rel=1e-12)
