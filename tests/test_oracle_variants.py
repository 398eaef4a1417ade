"""Pins of the oracle's paper variants: snapshots between steps (§2.2, the kick/drift equations
interpolating to output redshifts), the n_step sweep, and the CIC smoothing/alias correction of the
power spectrum (§3.3, Jing 2005) for a locally flat spectrum."""

import numpy as np
import pytest

import cola_inputs
from oracle import cic, cola, cosmology, fourier, power
from oracle.cosmology import Params

P = Params(np_side=8, nmesh=16, box=64.0)


def _state(seed=3, amp=0.7):
    rng = np.random.default_rng(seed)
    n = P.np_side ** 3
    psi1 = rng.standard_normal((3, n)) * amp
    psi2 = rng.standard_normal((3, n)) * amp * 0.2
    s = rng.standard_normal((3, n)) * amp
    v = rng.standard_normal((3, n)) * 0.1
    return s, v, psi1, psi2


@pytest.mark.parametrize("i", [1, 4, 9])
def test_snapshot_at_next_force_time_is_the_step(i):
    """a_snap = a_{i+1}: the partial drift is the whole drift, so the snapshot is step i's result."""
    s, v, psi1, psi2 = _state()
    c = cosmology.step_scalars(P, i)
    s1, v1 = cola.step(i, s, v, psi1, psi2, P)
    ss, vs = cola.snapshot(i, s, v, psi1, psi2, P, c["a_next"])
    np.testing.assert_allclose(ss, s1, rtol=0, atol=1e-10)
    np.testing.assert_allclose(vs, cola.final_velocity(v1, psi1, psi2, P, c["a_next"]), rtol=0, atol=1e-10)


def test_snapshot_at_the_force_time_has_not_moved():
    """a_snap = a_i: no drift and no 2LPT growth yet; only the velocity has been kicked."""
    s, v, psi1, psi2 = _state()
    c = cosmology.step_scalars(P, 5)
    ss, _ = cola.snapshot(5, s, v, psi1, psi2, P, c["a"])
    np.testing.assert_allclose(ss, s, rtol=0, atol=1e-12)


@pytest.mark.parametrize("a_snap", [0.55, 0.578, 0.6])
def test_snapshot_of_pure_2lpt_motion_is_the_2lpt_trajectory(a_snap):
    """With F_res = 0 and v_res = 0 the particles ride x_2LPT: s(a) = D1(a) Psi1 + D2(a) Psi2 and
    v = a^2 dx_2LPT/dt at any a_snap in [a_i, a_{i+1}] (§2.1)."""
    _, _, psi1, psi2 = _state(5)
    i = 5
    om = P.omega_m
    a_i = i / P.nstep
    s = cosmology.d1(a_i, om) * psi1 + cosmology.d2(a_i, om) * psi2

    def f2lpt(ss, fs):   # the exact 2LPT acceleration at a_i: F_res vanishes
        return fs * (cosmology.d1(a_i, om) * psi1 + (cosmology.d2(a_i, om) - cosmology.d1(a_i, om) ** 2) * psi2)

    ss, vs = cola.snapshot(i, s, np.zeros_like(s), psi1, psi2, P, a_snap, force=f2lpt)
    np.testing.assert_allclose(ss, cosmology.d1(a_snap, om) * psi1 + cosmology.d2(a_snap, om) * psi2,
                               rtol=0, atol=1e-12)
    f1, f2 = cosmology.lpt_velocity_factors(a_snap, om)
    np.testing.assert_allclose(vs, f1 * psi1 + f2 * psi2, rtol=1e-12, atol=1e-14)


def test_snapshot_drift_in_eds_is_the_closed_form():
    """Omega_m = 1: the partial drift integral of eq. (cola-drift) from a_i to a_snap is
    [a^(n - 1/2) / (n - 1/2)] / a_half^n (H = a^-3/2), so a free particle moves by that times v."""
    p = Params(np_side=8, nmesh=16, box=64.0, omega_m=1.0)
    i, a_snap = 3, 0.37
    c = cosmology.step_scalars(p, i)
    n = p.nlpt
    closed = (a_snap ** (n - 0.5) - c["a"] ** (n - 0.5)) / (n - 0.5) / c["a_hi"] ** n
    n3 = p.np_side ** 3
    v = np.ones((3, n3))
    zero = np.zeros((3, n3))
    ss, _ = cola.snapshot(i, zero, v, zero, zero, p, a_snap, force=lambda s, fs: np.zeros_like(s))
    np.testing.assert_allclose(ss, closed * v, rtol=1e-10)


def test_snapshot_rejects_times_outside_the_step():
    s, v, psi1, psi2 = _state()
    with pytest.raises(ValueError):
        cola.snapshot(3, s, v, psi1, psi2, P, 0.45)


@pytest.mark.parametrize("nstep", [20, 50, 100])
def test_more_steps_converge_to_the_same_free_motion(nstep):
    """n_step sweep (the paper varies the number of steps): the 2LPT-only trajectory (exact force
    F = F_2LPT) is independent of n_step and ends at D1(1) Psi1 + D2(1) Psi2."""
    p = Params(np_side=8, nmesh=16, box=64.0, nstep=nstep)
    _, _, psi1, psi2 = _state(7)
    s, v = cola.initial_state(psi1, psi2, p)
    for i in range(1, p.nstep + 1):
        c = cosmology.step_scalars(p, i)
        s, v = cola.step(i, s, v, psi1, psi2, p,
                         force=lambda ss, fs, c=c: c["c1"] * psi1 + c["c2"] * psi2)
    np.testing.assert_allclose(s, cosmology.d1(1.0, p.omega_m) * psi1 + cosmology.d2(1.0, p.omega_m) * psi2,
                               rtol=0, atol=1e-11)


# ---- CIC correction of P(k) -------------------------------------------------------------------
def _sinc(x):
    return np.sinc(x / np.pi)   # sin(x)/x


@pytest.mark.parametrize("m,n", [(0, 16), (3, 16), (8, 16), (5, 24), (11, 24)])
def test_cic_alias_sum_equals_brute_force(m, n):
    """C2 closed form against the alias sum of the textbook CIC window W = sinc^2(pi m / N), summed
    over 4001 aliases m + N j (the tail beyond is < 1e-9)."""
    j = np.arange(-2000, 2001)
    brute = np.sum(_sinc(np.pi * (m + n * j) / n) ** 4)
    closed = power.cic_alias_sum(np.array(m), np.array(0), np.array(0), n)
    assert closed == pytest.approx(brute, rel=1e-9)


def test_cic_correction_removes_shot_noise_of_a_random_field():
    """Uniform random (Poisson) particles: the raw CIC spectrum is (V/n) C2(k) mode by mode on
    average, so the corrected spectrum averages to zero (statistically, over all bins)."""
    rng = np.random.default_rng(11)
    n_side, nm, box = 24, 32, 100.0
    n = n_side ** 3
    x = rng.uniform(0.0, nm, size=(3, n))
    rho = cic.cic_exact_mesh(x, nm)
    delta = rho * (nm ** 3 / n) - 1.0
    _, praw, cnt = power.power_spectrum(delta, box, 16)
    _, pcor, _ = power.power_spectrum(delta, box, 16, cic_correct=True, n_particles=n)
    shot = box ** 3 / n
    sel = cnt > 50
    assert np.all(praw[sel] < shot)                     # the window suppresses it
    w = cnt[sel]
    assert abs(np.sum(pcor[sel] * w) / np.sum(w)) < 0.02 * shot
