"""Pins of the oracle's Fourier conventions and PM force (§2.2 Poisson equation, §2.3 PM mesh):
brute-force DFT, closed-form plane-wave force, momentum conservation, zero self-force and the
Newtonian limit of the pair force (Appendix A: correct beyond about 2.7 cells)."""

import numpy as np
import pytest

import cola_inputs
from oracle import cic, fourier, pm


@pytest.mark.parametrize("n", [6, 8, 10, 12, 15])
def test_library_fft_matches_naive_dft(n):
    x = cola_inputs.random_field((n, n, n), seed=n)
    full = fourier.naive_dft3(x)
    np.testing.assert_allclose(fourier.rfft3(x), full[:, :, : n // 2 + 1], atol=1e-10)


def test_mode_numbers_and_nyquist():
    assert list(fourier.mode_numbers(8)) == [0, 1, 2, 3, -4, -3, -2, -1]
    assert list(fourier.odd_mode(fourier.mode_numbers(8), 8)) == [0, 1, 2, 3, 0, -3, -2, -1]


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 1), (3, -1, 2)])
def test_plane_wave_force_closed_form(m):
    # delta = A cos(k.x): phi = -c delta / k^2; the 4-point central difference of phi along axis a,
    # (8 [phi(x+1) - phi(x-1)] - [phi(x+2) - phi(x-2)]) / 12, gives F_a = -c A (D_a / k^2) sin(k.x)
    # with D_a = (8 sin k_a - sin 2 k_a) / 6
    n, amp, c = 16, 0.3, 1.7
    g = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    k = [2 * np.pi * mi / n for mi in m]
    phase = sum(k[a] * g[a] for a in range(3))
    f = pm.force_mesh(amp * np.cos(phase), c)
    k2 = sum(ki * ki for ki in k)
    phi = -c * amp * np.cos(phase) / k2
    for a in range(3):
        fd = -(8 * (np.roll(phi, -1, a) - np.roll(phi, 1, a))
               - (np.roll(phi, -2, a) - np.roll(phi, 2, a))) / 12.0
        np.testing.assert_allclose(f[a], fd, atol=1e-13)
        da = (8 * np.sin(k[a]) - np.sin(2 * k[a])) / 6
        np.testing.assert_allclose(f[a], -c * amp * da / k2 * np.sin(phase), atol=1e-13)


def test_momentum_conservation_and_sum_of_forces():
    npd, nm = 8, 16
    s = cola_inputs.random_displacements(npd, seed=4, amplitude=3.0)
    f = pm.pm_force(s, npd, nm, 1.0)
    assert np.abs(f.sum(axis=1)).max() < 1e-12 * np.abs(f).sum()


@pytest.mark.parametrize("pos", [(3.3, 7.9, 1.2), (0.0, 0.5, 15.75)])
def test_self_force_vanishes(pos):
    nm = 16
    x = np.array(pos)[:, None]
    rho = cic.cic_exact_mesh(x, nm)
    delta = rho * nm ** 3 - 1.0
    fm = pm.force_mesh(delta, 1.0)
    c = np.floor(x).astype(int)
    w1 = x - c
    f = cic.cic_interp(fm, c, w1)
    assert np.abs(f).max() < 1e-12 * np.abs(fm).max()


def test_pair_force_tends_to_newtonian():
    # Appendix A: the PM force is correct beyond ~2.7 cells.  Mean radial force of a CIC particle
    # on CIC test particles at distance r (random placements and directions) against the
    # periodic Newtonian force near the source, -M/(4 pi r^2) + M r/(3V) (the second term is the
    # uniform neutralising background; cubic image lattice terms are O((r/L)^3)).
    nm = 32
    rng = np.random.default_rng(0)
    ratio = {}
    for r in (1.0, 3.0, 4.0):
        vals = []
        for _ in range(4):
            x0 = rng.uniform(0, nm, size=(3, 1))
            fm = pm.force_mesh(cic.cic_exact_mesh(x0, nm) * nm ** 3 - 1.0, 1.0)
            u = rng.normal(size=(3, 300))
            u /= np.linalg.norm(u, axis=0)
            x1 = x0 + r * u
            c = np.floor(x1).astype(int)
            fr = (cic.cic_interp(fm, c, x1 - c) * u).sum(axis=0)
            v = float(nm ** 3)
            vals.append(fr / (-v / (4 * np.pi * r * r) + v * r / (3 * v)))
        ratio[r] = float(np.mean(np.concatenate(vals)))
    assert ratio[1.0] < 0.9                      # softened inside a cell
    assert abs(ratio[3.0] - 1.0) < 0.03 and abs(ratio[4.0] - 1.0) < 0.02


# ---- the plane-wave closed forms used at full mesh size, pinned to the oracle's FFT path -----------
WAVES = [((1, 0, 0), 0.2, 0.3), ((3, -2, 5), 0.1, -1.1), ((-4, 5, 0), 0.15, 2.0), ((0, 0, 7), 0.05, 0.7),
         ((6, 7, -3), 0.1, -2.5)]


@pytest.mark.parametrize("n", [16, 18])
def test_plane_wave_closed_forms_match_the_fft_path(n):
    from oracle import fourier, pm
    cells = np.arange(n ** 3)
    delta = pm.plane_wave_density(WAVES, n, cells).reshape(n, n, n)
    dk = fourier.rfft3(delta)
    sparse = pm.plane_wave_spectrum(WAVES, n)
    expect = np.zeros_like(dk)
    for key, val in sparse.items():
        expect[key] = val
    np.testing.assert_allclose(dk, expect, atol=1e-9 * n ** 3)
    f = pm.force_mesh(delta, 1.37).reshape(3, -1)
    np.testing.assert_allclose(pm.plane_wave_force(WAVES, n, 1.37, cells), f, rtol=0, atol=1e-12)
    # a wave on the k_z = 0 plane is stored twice (+m and -m); others once
    assert ((-4) % n, 5, 0) in sparse and (4, (-5) % n, 0) in sparse
    assert (3, (-2) % n, 5) in sparse and ((-3) % n, 2, (-5) % n) not in sparse
