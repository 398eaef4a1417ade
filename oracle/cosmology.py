"""Oracle: FP64 background cosmology, growth factors, linear P(k) and COLA time coefficients.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed:
  * flat LCDM background, H0 = 1 units ........ §1 (cosmology), §2.2 (Poisson eq., eq. motion)
  * D1, D2 = -3/7 D1^2 Omega(a)^(-1/143) ....... §2.1 (2LPT growing mode and its footnote)
  * time grid a_i = i / n_step ................. §2.2, eq. (drift-a)
  * initial condition, paper and original ...... §2.2 eq. (initial_time); Appendix A eq. (initial_time_original)
  * drift factor ............................... §2.2 eq. (cola-drift) with the ansatz eq. (ansatz-drift)
  * kick factor ................................ §2.2 eq. (cola-kick) with the ansatz eq. (ansatz-kick)
  * constant-velocity drift ansatz (TZE) ....... §2.1 (the alternative ansatz v_res = const)
Readings where the paper is silent or garbled:
  * Omega(a) = Om / (Om + OL a^3): the printed formula lost its division.
  * the 2LPT acceleration uses the growth ODEs d/dt(a^2 dD1/dt) = 3/2 Om D1 / a and
    d/dt(a^2 dD2/dt) = 3/2 Om (D2 - D1^2) / a, which the paper does not write out.
  * P(k) = A k^ns T_BBKS(k)^2 with Gamma = Om h and A from sigma8 (8 Mpc/h top hat).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import integrate

_QUAD = dict(epsabs=0.0, epsrel=1e-13, limit=400)


@dataclasses.dataclass(frozen=True)
class Params:
    """Physical and numerical parameters of one COLA realisation (§2.2, §2.3)."""

    omega_m: float = 0.27
    h: float = 0.7
    n_s: float = 0.96
    sigma8: float = 0.8
    box: float = 256.0          # L in Mpc/h
    np_side: int = 32           # particles per side
    nmesh: int = 64             # PM mesh cells per side
    nstep: int = 10             # n_step of eq. (drift-a)
    nlpt: float = -2.5          # n_LPT of eq. (ansatz-kick)
    ic_mode: int = 0            # 0: eq. (initial_time); 1: eq. (initial_time_original)
    drift_ansatz: int = 0       # 0: eq. (ansatz-drift); 1: v_res constant during the drift

    @property
    def n(self) -> int:
        return self.np_side ** 3


# ---------------------------------------------------------------------------------------------
# Background and growth
# ---------------------------------------------------------------------------------------------

def hubble(a: float, om: float) -> float:
    """H(a)/H0 of a flat LCDM universe with Omega_Lambda = 1 - Om."""
    return math.sqrt(om / a ** 3 + (1.0 - om))


def dhubble_da(a: float, om: float) -> float:
    """dH/da of ``hubble``."""
    return -1.5 * om / a ** 4 / hubble(a, om)


def omega_of_a(a: float, om: float) -> float:
    """Matter density parameter at scale factor a (§2.1 footnote): Om / (Om + OL a^3)."""
    return om / (om + (1.0 - om) * a ** 3)


def _growth_integral(a: float, om: float) -> float:
    """int_0^a da' / (a' H(a'))^3, the integral of the growing mode."""
    if a <= 0.0:
        return 0.0
    val, _ = integrate.quad(lambda x: 1.0 / (x * hubble(x, om)) ** 3, 0.0, a, **_QUAD)
    return val


def d1(a: float, om: float) -> float:
    """Linear growth factor D1(a) = H(a) I(a) / (H(1) I(1)), normalised to D1(1) = 1 (§2.1)."""
    return hubble(a, om) * _growth_integral(a, om) / _growth_integral(1.0, om)


def d1_da(a: float, om: float) -> float:
    """dD1/da from differentiating H(a) I(a) / I(1)."""
    i1 = _growth_integral(1.0, om)
    return (dhubble_da(a, om) * _growth_integral(a, om)
            + hubble(a, om) / (a * hubble(a, om)) ** 3) / i1


def d2(a: float, om: float) -> float:
    """Second-order growth D2 = -3/7 D1^2 Omega(a)^(-1/143) (§2.1 and its footnote)."""
    return -3.0 / 7.0 * d1(a, om) ** 2 * omega_of_a(a, om) ** (-1.0 / 143.0)


def d2_da(a: float, om: float) -> float:
    """Analytic derivative of ``d2``."""
    ol = 1.0 - om
    om_a = omega_of_a(a, om)
    domega = -3.0 * om * ol * a ** 2 / (om + ol * a ** 3) ** 2
    g1, g1p = d1(a, om), d1_da(a, om)
    return -3.0 / 7.0 * (2.0 * g1 * g1p * om_a ** (-1.0 / 143.0)
                         + g1 ** 2 * (-1.0 / 143.0) * om_a ** (-1.0 / 143.0 - 1.0) * domega)


# ---------------------------------------------------------------------------------------------
# COLA time coefficients, eqs. (cola-drift) and (cola-kick)
# ---------------------------------------------------------------------------------------------

def drift_factor(a0: float, a1: float, a_half: float, om: float, nlpt: float,
                 ansatz: int = 0) -> float:
    """Drift integral of eq. (cola-drift): int_{t(a0)}^{t(a1)} (a/a_half)^nLPT dt / a^2.

    With dt = da / (a H) this is int_{a0}^{a1} (a/a_half)^nLPT / (a^3 H(a)) da.  ansatz=1 is the
    constant residual velocity of §2.1, which drops the (a/a_half)^nLPT factor.
    """
    if ansatz == 0:
        f = lambda a: (a / a_half) ** nlpt / (a ** 3 * hubble(a, om))
    else:
        f = lambda a: 1.0 / (a ** 3 * hubble(a, om))
    val, _ = integrate.quad(f, a0, a1, **_QUAD)
    return val


def kick_factor(a_lo: float, a_hi: float, a_i: float, om: float, nlpt: float) -> float:
    """Kick factor of eq. (cola-kick): (a_hi^n - a_lo^n) / (n a_i^(n-1) adot(a_i)), adot = a H."""
    n = nlpt
    return (a_hi ** n - a_lo ** n) / (n * a_i ** (n - 1.0) * a_i * hubble(a_i, om))


def step_scalars(p: Params, i: int) -> dict:
    """Every scalar of COLA step i (1-based): force at a_i, kick a_lo -> a_hi, drift a_i -> a_{i+1}.

    Schedule (§2.2): a_i = i/n_step, half steps a_{i+1/2} = (i+1/2)/n_step.  Positions start at
    a_1 from 2LPT.  ic_mode 0 (eq. initial_time) starts the residual velocity at a_{1/2}; ic_mode 1
    (eq. initial_time_original) at a_1.  The last step kicks to a_{n_step} and does not drift.
    """
    ns = p.nstep
    om, nl = p.omega_m, p.nlpt
    a_i = i / ns
    a_lo = (i - 0.5) / ns
    if i == 1 and p.ic_mode == 1:
        a_lo = a_i
    last = i == ns
    a_hi = a_i if last else (i + 0.5) / ns
    g1, g2 = d1(a_i, om), d2(a_i, om)
    pref = 1.5 * om / a_i                              # (3/2) Om / a of the Poisson equation, §2.2
    out = dict(a=a_i, a_lo=a_lo, a_hi=a_hi,
               force_scale=pref,
               c1=pref * g1,                           # 2LPT acceleration, first order
               c2=pref * (g2 - g1 * g1),               # 2LPT acceleration, second order
               kick=kick_factor(a_lo, a_hi, a_i, om, nl))
    if last:
        out.update(drift=0.0, dd1=0.0, dd2=0.0, a_next=a_i)
    else:
        a_n = (i + 1) / ns
        out.update(drift=drift_factor(a_i, a_n, (i + 0.5) / ns, om, nl, p.drift_ansatz),
                   dd1=d1(a_n, om) - g1, dd2=d2(a_n, om) - g2, a_next=a_n)
    return out


def lpt_velocity_factors(a: float, om: float) -> tuple[float, float]:
    """a^2 dD1/dt and a^2 dD2/dt (dt = da / (a H)): the canonical 2LPT velocity factors."""
    f = a ** 3 * hubble(a, om)
    return f * d1_da(a, om), f * d2_da(a, om)


# ---------------------------------------------------------------------------------------------
# Linear power spectrum, BBKS transfer function and sigma8 normalisation
# ---------------------------------------------------------------------------------------------

def t_bbks(k, om: float, h: float):
    """BBKS transfer function with Gamma = Om h, k in h/Mpc (no baryon correction)."""
    k = np.asarray(k, dtype=np.float64)
    q = k / (om * h)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (np.log1p(2.34 * q) / (2.34 * q)
             * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)
    return np.where(q > 0, t, 1.0)


def tophat_window(x):
    """Fourier transform of a unit top hat, 3 (sin x - x cos x) / x^3 (series for small x)."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1e-3
    xs = np.where(small, 1.0, x)
    w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return np.where(small, 1.0 - x * x / 10.0, w)


def _bbks_shape(p: Params):
    """k -> k^ns T_BBKS(k)^2, the shape of the linear spectrum before its amplitude."""
    return lambda k: k ** p.n_s * t_bbks(k, p.omega_m, p.h) ** 2


def sigma2_of(power, radius: float = 8.0) -> float:
    """sigma^2(R) = (1/2pi^2) int k^2 P(k) W(kR)^2 dk for a spectrum P(k) (k in h/Mpc), by adaptive
    quadrature in ln k over [1e-7, 1e3] h/Mpc."""
    def integrand(lnk: float) -> float:
        k = math.exp(lnk)
        return k ** 3 * float(power(k)) * float(tophat_window(k * radius)) ** 2 / (2.0 * math.pi ** 2)
    val, _ = integrate.quad(integrand, math.log(1e-7), math.log(1e3), epsabs=0.0, epsrel=1e-12, limit=2000)
    return val


def sigma2_of_simpson(power, radius: float = 8.0, npts: int = 400001) -> float:
    """The same integral by composite Simpson on a uniform ln k grid (an independent quadrature)."""
    lnk = np.linspace(math.log(1e-7), math.log(1e3), npts)
    k = np.exp(lnk)
    f = k ** 3 * power(k) * tophat_window(k * radius) ** 2 / (2.0 * math.pi ** 2)
    return float(integrate.simpson(f, x=lnk))


def sigma2_quad(amp: float, p: Params, radius: float = 8.0) -> float:
    """sigma^2(R) of P(k) = amp k^ns T_BBKS(k)^2 (adaptive quadrature)."""
    shape = _bbks_shape(p)
    return sigma2_of(lambda k: amp * shape(k), radius)


def sigma2_simpson(amp: float, p: Params, radius: float = 8.0, npts: int = 400001) -> float:
    """sigma^2(R) of P(k) = amp k^ns T_BBKS(k)^2 (composite Simpson)."""
    shape = _bbks_shape(p)
    return sigma2_of_simpson(lambda k: amp * shape(k), radius, npts)


def power_amplitude(p: Params) -> float:
    """A such that P(k) = A k^ns T(k)^2 has sigma(8 Mpc/h) = sigma8 at a = 1."""
    return p.sigma8 ** 2 / sigma2_quad(1.0, p)


def linear_power(k, p: Params, amp: float | None = None):
    """Linear matter power spectrum at a = 1 in (Mpc/h)^3, k in h/Mpc."""
    if amp is None:
        amp = power_amplitude(p)
    k = np.asarray(k, dtype=np.float64)
    return amp * k ** p.n_s * t_bbks(k, p.omega_m, p.h) ** 2
