"""Pins of the oracle's background cosmology, growth factors, P(k) normalisation and COLA
time coefficients (§2.1, §2.2) against closed forms, an ODE integration and an independent
quadrature."""

import math

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology as C
from oracle.cosmology import Params

EDS = 1.0 - 1e-15   # Omega_m -> 1 (Einstein-de Sitter); Omega_Lambda ~ 0


@pytest.mark.parametrize("a", [0.05, 0.1, 0.37, 0.8, 1.0])
def test_eds_growth_closed_forms(a):
    # EdS: H = a^-3/2, D1 = a, D2 = -3/7 a^2 (Omega(a) = 1), dD1/da = 1
    assert C.hubble(a, 1.0) == pytest.approx(a ** -1.5, rel=1e-14)
    assert C.d1(a, EDS) == pytest.approx(a, rel=1e-11)
    assert C.d1_da(a, EDS) == pytest.approx(1.0, rel=1e-10)
    assert C.d2(a, EDS) == pytest.approx(-3.0 / 7.0 * a * a, rel=1e-10)
    assert C.d2_da(a, EDS) == pytest.approx(-6.0 / 7.0 * a, rel=1e-10)


@pytest.mark.parametrize("i", [1, 2, 5, 9])
@pytest.mark.parametrize("nlpt", [-2.5, -1.0, 0.7])
def test_eds_drift_and_kick_closed_forms(i, nlpt):
    # drift: int a^n / a_h^n * a^-3/2 da = [a^(n-1/2)/(n-1/2)] / a_h^n ;  kick: n a^(n-1) adot = n a^n a^-3/2
    ns = 10
    a0, a1, ah = i / ns, (i + 1) / ns, (i + 0.5) / ns
    closed = (a1 ** (nlpt - 0.5) - a0 ** (nlpt - 0.5)) / (nlpt - 0.5) / ah ** nlpt
    assert C.drift_factor(a0, a1, ah, 1.0, nlpt) == pytest.approx(closed, rel=1e-12)
    alo, ahi, ai = (i - 0.5) / ns, (i + 0.5) / ns, i / ns
    kclosed = (ahi ** nlpt - alo ** nlpt) / (nlpt * ai ** nlpt * ai ** -1.5)
    assert C.kick_factor(alo, ahi, ai, 1.0, nlpt) == pytest.approx(kclosed, rel=1e-13)


def test_lcdm_growth_matches_ode_integration():
    # D'' + (3/a + H'/H) D' - 3/2 Om / (a^5 H^2) D = 0, growing mode D ~ a deep in matter era
    om = 0.27

    def rhs(a, y):
        d, dp = y
        h = C.hubble(a, om)
        return [dp, -(3.0 / a + C.dhubble_da(a, om) / h) * dp + 1.5 * om / (a ** 5 * h * h) * d]

    a0 = 1e-4
    sol = integrate.solve_ivp(rhs, (a0, 1.0), [a0, 1.0], rtol=1e-12, atol=1e-16, dense_output=True)
    d_one = sol.sol(1.0)[0]
    for a in (0.05, 0.1, 0.3, 0.6, 0.9):
        assert C.d1(a, om) == pytest.approx(sol.sol(a)[0] / d_one, rel=1e-8)
        assert C.d1_da(a, om) == pytest.approx(sol.sol(a)[1] / d_one, rel=1e-7)


@pytest.mark.parametrize("a", [0.07, 0.3, 0.95])
def test_growth_derivatives_match_finite_differences(a):
    om, h = 0.27, 1e-5
    fd1 = (C.d1(a + h, om) - C.d1(a - h, om)) / (2 * h)
    fd2 = (C.d2(a + h, om) - C.d2(a - h, om)) / (2 * h)
    assert C.d1_da(a, om) == pytest.approx(fd1, rel=1e-8)
    assert C.d2_da(a, om) == pytest.approx(fd2, rel=1e-8)


def test_omega_of_a_limits():
    om = 0.27
    assert C.omega_of_a(1.0, om) == pytest.approx(om, rel=1e-15)
    assert C.omega_of_a(1e-4, om) == pytest.approx(1.0, abs=1e-10)
    # Omega(a) = Om a^-3 / H(a)^2 by definition of the matter fraction
    for a in (0.2, 0.5):
        assert C.omega_of_a(a, om) == pytest.approx(om / a ** 3 / C.hubble(a, om) ** 2, rel=1e-14)


def test_sigma8_normalisation_two_quadratures():
    p = Params()
    amp = C.power_amplitude(p)
    assert C.sigma2_simpson(amp, p) == pytest.approx(p.sigma8 ** 2, rel=1e-9)


def test_bbks_limits():
    om, h = 0.27, 0.7
    assert float(C.t_bbks(1e-7, om, h)) == pytest.approx(1.0, abs=1e-5)
    # large q: the bracket tends to (6.71 q)^4, so T -> ln(2.34 q) / (2.34 q) / (6.71 q)
    k = 1e5
    q = k / (om * h)
    assert float(C.t_bbks(k, om, h)) == pytest.approx(math.log(2.34 * q) / (2.34 * q) / (6.71 * q),
                                                      rel=1e-3)
    ks = np.logspace(-4, 2, 200)
    t = C.t_bbks(ks, om, h)
    assert np.all(np.diff(t) < 0)


def test_tophat_window_series_and_zero():
    # W(x) = 3 j1(x) / x; first zero of tan x = x at x = 4.493409457909064
    assert float(C.tophat_window(4.493409457909064)) == pytest.approx(0.0, abs=1e-12)
    assert float(C.tophat_window(1e-4)) == pytest.approx(1.0 - 1e-9, abs=1e-15)


def test_small_steps_reduce_to_leapfrog():
    # eq. (leapfrog1/2): for short steps the kick tends to dt and the drift to dt / a^2
    om, nl = 0.27, -2.5
    ai, eps = 0.5, 1e-5
    dt = integrate.quad(lambda a: 1.0 / (a * C.hubble(a, om)), ai - eps, ai + eps,
                        epsabs=0, epsrel=1e-13)[0]
    assert C.kick_factor(ai - eps, ai + eps, ai, om, nl) == pytest.approx(dt, rel=1e-8)
    assert C.drift_factor(ai - eps, ai + eps, ai, om, nl) == pytest.approx(dt / ai ** 2, rel=1e-8)


def test_step_schedule():
    p = Params(nstep=10)
    first = C.step_scalars(p, 1)
    assert (first["a"], first["a_lo"], first["a_hi"]) == (0.1, 0.05, 0.15)
    orig = C.step_scalars(Params(nstep=10, ic_mode=1), 1)
    assert orig["a_lo"] == 0.1
    last = C.step_scalars(p, 10)
    assert (last["a"], last["a_lo"], last["a_hi"]) == (1.0, 0.95, 1.0)
    assert last["drift"] == 0.0 and last["dd1"] == 0.0 and last["dd2"] == 0.0
    # the 2LPT acceleration coefficients: (3/2) Om/a [D1, D2 - D1^2]
    assert first["c1"] == pytest.approx(1.5 * 0.27 / 0.1 * C.d1(0.1, 0.27), rel=1e-15)
    # D1 increments telescope to D1(1) - D1(a_1)
    tot = sum(C.step_scalars(p, i)["dd1"] for i in range(1, 11))
    assert tot == pytest.approx(1.0 - C.d1(0.1, 0.27), rel=1e-12)


def test_constant_drift_ansatz():
    # ansatz 1 drops the (a/a_half)^n factor: equals the nlpt = 0 drift of ansatz 0
    om = 0.27
    a = C.drift_factor(0.3, 0.4, 0.35, om, -2.5, ansatz=1)
    b = C.drift_factor(0.3, 0.4, 0.35, om, 0.0, ansatz=0)
    assert a == pytest.approx(b, rel=1e-13)


# ---- outside pins of the linear spectrum: the BBKS coefficients and the sigma^2 integral ----------

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def bbks_golden():
    """The five published BBKS coefficients (tests/golden/bbks_transfer.txt, with its citation)."""
    c = {}
    for line in open(__import__("os").path.join(GOLDEN, "bbks_transfer.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()
            c[name] = float(value)
    return c


def bbks_from_golden(q):
    """T(q) evaluated term by term from the golden coefficients (log-sum form, not the oracle's)."""
    c = bbks_golden()
    q = np.asarray(q, dtype=np.float64)
    poly = 1.0 + c["c1"] * q + (c["c2"] * q) ** 2 + (c["c3"] * q) ** 3 + (c["c4"] * q) ** 4
    return np.exp(np.log(np.log1p(c["c0"] * q)) - np.log(c["c0"] * q) - 0.25 * np.log(poly))


@pytest.mark.parametrize("om,h", [(0.27, 0.7), (0.3, 0.67), (1.0, 0.5)])
def test_bbks_matches_the_published_coefficients(om, h):
    # interior q, where every coefficient matters: a one-digit change of any of them moves T by
    # more than 5e-5 somewhere on this grid
    q = np.logspace(-3, 2, 61)
    k = q * om * h
    np.testing.assert_allclose(C.t_bbks(k, om, h), bbks_from_golden(q), rtol=1e-13)


def test_bbks_typos_are_visible_to_the_pin():
    """Each coefficient, changed in its last printed digit, moves T by > 5e-5 somewhere in q (far
    above the pin's 1e-13)."""
    c = bbks_golden()
    q = np.logspace(-3, 2, 61)

    def t(cc):
        poly = 1.0 + cc["c1"] * q + (cc["c2"] * q) ** 2 + (cc["c3"] * q) ** 3 + (cc["c4"] * q) ** 4
        return np.log1p(cc["c0"] * q) / (cc["c0"] * q) * poly ** -0.25

    base = t(c)
    for name, step in (("c0", 0.01), ("c1", 0.01), ("c2", 0.1), ("c3", 0.01), ("c4", 0.01)):
        cc = dict(c)
        cc[name] += step
        assert np.max(np.abs(t(cc) / base - 1.0)) > 5e-5, name


def test_bbks_shape_agrees_with_eisenstein_hu_zero_baryon():
    """An independent fit to the same CDM physics: Eisenstein & Hu 1998 (ApJ 496, 605) eqs. (28)-(29)
    without baryons, T0 = L0 / (L0 + C0 q^2), L0 = ln(2e + 1.8 q), C0 = 14.2 + 731 / (1 + 62.5 q),
    with q = k / (Gamma h Mpc^-1) at Theta_2.7 = 1.  The two fits agree to 4% from q = 1e-3 to 30;
    a wrong power, a swapped coefficient or a dropped term breaks that."""
    om, h = 0.27, 0.7
    q = np.logspace(-3, 1.5, 91)
    l0 = np.log(2.0 * math.e + 1.8 * q)
    c0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    t_eh = l0 / (l0 + c0 * q * q)
    ratio = C.t_bbks(q * om * h, om, h) / t_eh
    assert np.max(np.abs(ratio - 1.0)) < 0.045


def _power_law(amp, n):
    return lambda k: amp * np.asarray(k, dtype=np.float64) ** n


@pytest.mark.parametrize("radius", [5.0, 8.0])
def test_sigma2_of_power_laws_matches_real_space_closed_forms(radius):
    """sigma^2(R) of P = A k^n with a top hat, from real space: sigma^2 = <xi(|x - y|)> over pairs of
    points of the ball.  For n = -2, xi = A / (4 pi r); for n = -1, xi = A / (2 pi^2 r^2).  Two
    uniform points in a ball of radius R have <1/r> = 6 / (5R) and <1/r^2> = 9 / (4 R^2) (from their
    distance density 3 r^2/R^3 (1 - 3r/(4R) + r^3/(16 R^3)) on [0, 2R]), so sigma^2 = 3A / (10 pi R)
    and 9A / (8 pi^2 R^2).  This pins the 1/(2 pi^2) factor, the k^2 dk measure and the window."""
    amp = 3.7
    cases = ((-2.0, 3.0 * amp / (10.0 * math.pi * radius), 2e-6),   # the low-k cut leaves ~5e-7
             (-1.0, 9.0 * amp / (8.0 * math.pi ** 2 * radius ** 2), 1e-7))
    for n, closed, tol in cases:
        assert C.sigma2_of(_power_law(amp, n), radius) == pytest.approx(closed, rel=tol)
        assert C.sigma2_of_simpson(_power_law(amp, n), radius) == pytest.approx(closed, rel=tol)


def test_sigma2_of_white_noise_is_the_inverse_volume():
    """P = A (white noise): the mean over a ball of volume V has variance A / V (Parseval), less the
    part of the integral beyond the upper limit k = 1e3 h/Mpc, 9 A / (4 pi^2 R^3 X) with X = 1e3 R
    (the window's tail 9 cos^2 x / x^4 averaged)."""
    amp, radius = 2.0, 8.0
    x_max = 1e3 * radius
    expected = 3.0 * amp / (4.0 * math.pi * radius ** 3) - 9.0 * amp / (4.0 * math.pi ** 2 * radius ** 3 * x_max)
    assert C.sigma2_of(_power_law(amp, 0.0), radius) == pytest.approx(expected, rel=2e-6)
