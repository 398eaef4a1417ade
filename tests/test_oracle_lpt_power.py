"""Pins of the oracle's 2LPT (§2.1 growing mode, §2.3 2LPTic initial conditions) and of the power
spectrum estimator (§3.3): closed forms for plane waves, the divergence identity, the white-noise
variance and mode selection by brute force."""

import numpy as np
import pytest

import cola_inputs
from oracle import cosmology, fourier, lpt, power
from oracle.cosmology import Params


def _plane_wave_dk(n, waves):
    """Half spectrum of sum_j A_j cos(2 pi m_j . q / n) (computed by the library FFT)."""
    g = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    d = np.zeros((n, n, n))
    for amp, m in waves:
        d += amp * np.cos(2 * np.pi * sum(m[a] * g[a] for a in range(3)) / n)
    return fourier.rfft3(d), g


def test_zeldovich_plane_wave_first_order():
    # delta_L = A cos(k x) -> Psi1_x = -(A/k) sin(k x), Psi1_y = Psi1_z = 0
    n, box, amp = 16, 100.0, 0.4
    dk, g = _plane_wave_dk(n, [(amp, (2, 0, 0))])
    k = 2 * np.pi * 2 / box
    psi = lpt.first_order(dk, n, box)
    x = g[0] * box / n
    np.testing.assert_allclose(psi[0], -(amp / k) * np.sin(k * x), atol=1e-12)
    assert np.abs(psi[1:]).max() < 1e-12


def test_single_plane_wave_has_no_second_order_source():
    n, box = 16, 100.0
    dk, _ = _plane_wave_dk(n, [(0.4, (1, 2, 3))])
    assert np.abs(lpt.second_order_source(dk, n, box)).max() < 1e-14


def test_two_orthogonal_plane_waves_closed_form():
    # delta = A cos(k1 x) + B cos(k2 y): S = A B cos(k1 x) cos(k2 y),
    # Psi2 = grad phi2 with phi2 = -S / (k1^2 + k2^2)
    n, box, a_amp, b_amp = 16, 80.0, 0.3, -0.2
    dk, g = _plane_wave_dk(n, [(a_amp, (1, 0, 0)), (b_amp, (0, 3, 0))])
    k1, k2 = 2 * np.pi / box, 2 * np.pi * 3 / box
    x, y = g[0] * box / n, g[1] * box / n
    s = a_amp * b_amp * np.cos(k1 * x) * np.cos(k2 * y)
    np.testing.assert_allclose(lpt.second_order_source(dk, n, box), s, atol=1e-14)
    psi2 = lpt.second_order(dk, n, box)
    kk = k1 * k1 + k2 * k2
    np.testing.assert_allclose(psi2[0], a_amp * b_amp * k1 * np.sin(k1 * x) * np.cos(k2 * y) / kk,
                               atol=1e-13)
    np.testing.assert_allclose(psi2[1], a_amp * b_amp * k2 * np.cos(k1 * x) * np.sin(k2 * y) / kk,
                               atol=1e-13)
    assert np.abs(psi2[2]).max() < 1e-14


def test_divergence_of_psi1_is_minus_delta():
    # away from the Nyquist planes, i k . Psi1(k) = -delta_L(k)
    p = Params(box=200.0, np_side=16, nmesh=32)
    w = cola_inputs.white_noise(16, seed=7)
    dk = lpt.linear_density_k(w, p)
    psi = lpt.first_order(dk, 16, p.box)
    mx, my, mz = fourier.mode_grids(16)
    kf = 2 * np.pi / p.box
    div = sum(1j * kf * m * fourier.rfft3(psi[a]) for a, m in enumerate((mx, my, mz)))
    nyq = (np.abs(mx) == 8) | (np.abs(my) == 8) | (mz == 8)
    nyq = np.broadcast_to(nyq, dk.shape)
    np.testing.assert_allclose(div[~nyq], -dk[~nyq], atol=1e-10 * np.abs(dk).max())


def test_white_noise_variance_matches_sum_of_power():
    # E[delta_L(q)^2] = (1/V) sum_{k != 0} P(k) for unit white noise (the amplitude convention)
    p = Params(box=300.0, np_side=16, nmesh=32)
    amp = cosmology.power_amplitude(p)
    mx, my, mz = fourier.mode_grids(16)
    kmag = np.sqrt((mx * mx + my * my + mz * mz).astype(float)) * 2 * np.pi / p.box
    full_m = fourier.mode_numbers(16)
    km = np.sqrt(full_m[:, None, None] ** 2 + full_m[None, :, None] ** 2
                 + full_m[None, None, :] ** 2) * 2 * np.pi / p.box
    expect = cosmology.linear_power(km[km > 0], p, amp).sum() / p.box ** 3
    var = []
    for seed in range(40):
        dk = lpt.linear_density_k(cola_inputs.white_noise(16, seed=1000 + seed), p)
        var.append(np.mean(fourier.irfft3(dk, 16) ** 2))
    assert np.mean(var) == pytest.approx(expect, rel=0.03)
    assert kmag.shape == (16, 16, 9)


def test_half_space_selects_one_of_each_conjugate_pair():
    n = 10
    mask = power.half_space_mask(n)
    m = fourier.mode_numbers(n)
    sel = set()
    for i in range(n):
        for j in range(n):
            for kz in range(n // 2 + 1):
                if mask[i, j, kz]:
                    sel.add((m[i], m[j], kz))
    for mx in range(-n // 2 + 1, n // 2):
        for my in range(-n // 2 + 1, n // 2):
            for mz in range(-n // 2 + 1, n // 2):
                if (mx, my, mz) == (0, 0, 0):
                    continue
                a, b = (mx, my, mz) in sel, (-mx, -my, -mz) in sel
                assert a != b, (mx, my, mz)


def test_single_mode_power_and_bins():
    # delta = A cos(k.x) puts V A^2 / 4 in one selected mode
    n, box, amp, nb = 16, 160.0, 0.2, 8
    g = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    m = (2, -1, 3)
    d = amp * np.cos(2 * np.pi * sum(m[a] * g[a] for a in range(3)) / n)
    k, pk, cnt = power.power_spectrum(d, box, nb)
    m2 = 14
    edges = power.bin_edges_m2(n, nb)
    b = int(np.searchsorted(edges, m2, side="right") - 1)
    assert pk[b] * cnt[b] == pytest.approx(box ** 3 * amp ** 2 / 4, rel=1e-12)
    assert np.all(pk[np.arange(nb) != b] < 1e-25)


def test_bin_edges():
    e = power.bin_edges_m2(64, 64)
    assert e[0] == 1 and e[-1] == 32 * 32 and e[32] == 32
    assert np.all(np.diff(e) >= 0)
    # mode counts: every mode with 0 < |m| < N/2 lands in exactly one bin, once per conjugate pair
    n = 12
    _, _, cnt = power.power_spectrum(np.zeros((n, n, n)), 100.0, 6)
    full = fourier.mode_numbers(n)
    m2 = full[:, None, None] ** 2 + full[None, :, None] ** 2 + full[None, None, :] ** 2
    assert cnt.sum() * 2 == int(((m2 > 0) & (m2 < (n // 2) ** 2)).sum())
