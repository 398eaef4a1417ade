"""Pins of the oracle's COLA integrator (§2.1 residual decomposition, §2.2 eqs. cola-kick and
cola-drift): the Zel'dovich plane wave before shell crossing, linear growth at tiny amplitude,
momentum conservation and free streaming."""

import numpy as np
import pytest

import cola_inputs
from oracle import cic, cola, cosmology, fourier
from oracle.cosmology import Params


def _plane_wave_psi1(npd, nmesh, amp_cells):
    """Psi1_x = -A sin(2 pi x_q / N): the 1D Zel'dovich displacement of a cosine density mode."""
    q = cic.lattice_indices(npd).astype(np.float64)
    psi1 = np.zeros((3, npd ** 3))
    psi1[0] = -amp_cells * np.sin(2 * np.pi * q[0] / npd)
    return psi1, np.zeros_like(psi1)


def _run_plane_wave(npd, nmesh, force=None):
    amp = 0.08 * nmesh            # max |d s / d x| = 2 pi 0.08 D1 < 1: no shell crossing by a = 1
    p = Params(np_side=npd, nmesh=nmesh, box=100.0)
    psi1, psi2 = _plane_wave_psi1(npd, nmesh, amp)
    s, v = cola.initial_state(psi1, psi2, p)
    for i in range(1, p.nstep + 1):
        s, v = cola.step(i, s, v, psi1, psi2, p, force=force)
    return s, v, psi1 * cosmology.d1(1.0, p.omega_m), amp


def test_zeldovich_with_exact_gauss_force_stays_on_2lpt():
    # 1D before shell crossing Gauss's law gives F = (3/2)(Om/a)(x - q) exactly; then
    # F_res = (3/2)(Om/a) x_res, and x_res = v_res = 0 must persist through every kick and drift.
    s, v, lin, _ = _run_plane_wave(8, 16, force=lambda s, c: c * s)
    np.testing.assert_allclose(s, lin, atol=1e-13)
    assert np.abs(v).max() < 1e-14


def test_zeldovich_pm_error_shrinks_with_resolution():
    errs = []
    for npd, nmesh in ((16, 32), (32, 64)):
        s, _, lin, amp = _run_plane_wave(npd, nmesh)
        errs.append(np.abs(s - lin).max() / amp)
    assert errs[0] < 0.2 and errs[1] < 0.6 * errs[0]


def test_tiny_amplitude_follows_linear_growth_at_low_k():
    # sigma8 = 0.02: the fundamental lattice modes of s(a=1) follow D1 Psi1 + D2 Psi2.  What remains
    # is the PM discreteness of an r = 2 CIC lattice (aliases near the mesh Nyquist feed the force of
    # low modes at the per-cent level); it shrinks as the mesh is refined.
    def low_k_deviation(npd, nmesh):
        p = Params(sigma8=0.02, np_side=npd, nmesh=nmesh, box=12.5 * npd)
        out = cola.run(cola_inputs.white_noise(npd, seed=3), p)
        lin = (cosmology.d1(1.0, p.omega_m) * out["psi1"]
               + cosmology.d2(1.0, p.omega_m) * out["psi2"])
        mx, my, mz = fourier.mode_grids(npd)
        low = np.broadcast_to((mx * mx + my * my + mz * mz) == 1, (npd, npd, npd // 2 + 1))
        num = den = 0.0
        for a in range(3):
            dk = fourier.rfft3((out["s"][a] - lin[a]).reshape((npd,) * 3))
            lk = fourier.rfft3(lin[a].reshape((npd,) * 3))
            num += np.sum(np.abs(dk[low]) ** 2)
            den += np.sum(np.abs(lk[low]) ** 2)
        return np.sqrt(num / den)

    coarse, fine = low_k_deviation(16, 32), low_k_deviation(32, 64)
    assert fine < 0.04 and fine < 0.6 * coarse


def test_momentum_of_residual_velocity_is_conserved():
    p = Params(np_side=16, nmesh=32, box=200.0)
    out = cola.run(cola_inputs.white_noise(16, seed=4), p)
    scale = np.abs(out["v_res"]).sum()
    assert np.abs(out["v_res"].sum(axis=1)).max() < 1e-10 * scale


def test_free_streaming_uses_drift_integrals():
    # a uniform r = 1 lattice shifted as a whole has delta = 0, so F = 0; with Psi = 0 only v_res
    # moves s, by exactly the sum of the drift integrals
    p = Params(np_side=8, nmesh=8, box=50.0)
    zero = np.zeros((3, 8 ** 3))
    v0 = np.full((3, 8 ** 3), 0.125)
    s, v = zero.copy(), v0.copy()
    expect = 0.0
    for i in range(1, p.nstep + 1):
        s, v = cola.step(i, s, v, zero, zero, p)
        expect += cosmology.step_scalars(p, i)["drift"] * 0.125
    np.testing.assert_allclose(v, v0, atol=1e-15)
    np.testing.assert_allclose(s, expect, rtol=1e-14)
