"""Oracle: the COLA integrator (kick-drift in residual variables) and a whole realisation.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages:
  * residual decomposition x_res = x - x_2LPT, v_res = v - a^2 dx_2LPT/dt,
    F_res = F - d/dt(a^2 dx_2LPT/dt) ............................................ §2.1
  * x_2LPT = q + D1 Psi1 + D2 Psi2 ............................................... §2.1
  * kick v_res_{i-1/2} -> v_res_{i+1/2} with F_res(x_i) ........................ §2.2 eq. (cola-kick)
  * drift x_i -> x_{i+1} with v_res_{i+1/2} ..................................... §2.2 eq. (cola-drift)
  * schedule a_i = i / n_step, initial condition ................................ §2.2 eqs. (drift-a), (initial_time)

State: s = x - q (total displacement, PM cells), v_res (canonical, PM cells per unit time,
H0 = 1).  The 2LPT acceleration is F_2LPT = (3/2)(Om/a)[D1 Psi1 + (D2 - D1^2) Psi2]
(a reading: the paper names x_2LPT's acceleration without writing it; this follows from the 2LPT
growth equations).  The final kick ends at a_{n_step} and the last step does not drift (§2.2,
eq. drift-a: positions at a_i = i/n_step, velocities at the half steps).
"""

from __future__ import annotations

import numpy as np

from . import cosmology, lpt, pm, power


def initial_state(psi1, psi2, p: cosmology.Params):
    """s at a_1 from 2LPT (x_res = 0) and v_res = 0 (eq. initial_time / initial_time_original)."""
    a1 = 1.0 / p.nstep
    s = cosmology.d1(a1, p.omega_m) * psi1 + cosmology.d2(a1, p.omega_m) * psi2
    return s, np.zeros_like(s)


def step(i: int, s, v, psi1, psi2, p: cosmology.Params, force=None):
    """One COLA step i (1-based) in FP64: force at a_i, kick, then drift to a_{i+1}.

    Inputs may be float32; they are promoted to float64.  Returns (s, v) after the step.
    ``force(s, force_scale)`` replaces the PM force (tests use exact forces); the default is the
    particle-mesh force of ``pm.pm_force``.
    """
    c = cosmology.step_scalars(p, i)
    s = np.asarray(s, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    psi1 = np.asarray(psi1, dtype=np.float64)
    psi2 = np.asarray(psi2, dtype=np.float64)
    if force is None:
        f = pm.pm_force(s, p.np_side, p.nmesh, c["force_scale"])
    else:
        f = force(s, c["force_scale"])
    f_res = f - (c["c1"] * psi1 + c["c2"] * psi2)
    v = v + c["kick"] * f_res
    s = s + c["drift"] * v + c["dd1"] * psi1 + c["dd2"] * psi2
    return s, v


def snapshot(i: int, s, v, psi1, psi2, p: cosmology.Params, a_snap: float, force=None):
    """Positions and canonical velocities at a_snap between the force times a_i and a_{i+1}
    (§2.2: the kick/drift equations also interpolate between steps), from the state (s_i, v_res at
    a_{i-1/2}) before step i: kick as in ``step``, then the drift of eq. (cola-drift) and the 2LPT
    growth taken only up to a_snap.  The residual velocity between kicks is v_res(a_{i+1/2})
    (a reading: the paper's remark that an acceleration term could improve this is not applied).
    a_i <= a_snap <= a_{i+1} (a_snap = a_i = 1 after the last step)."""
    c = cosmology.step_scalars(p, i)
    a_i = c["a"]
    if not (a_i - 1e-12 <= a_snap <= c["a_next"] + 1e-12):
        raise ValueError("a_snap outside [a_i, a_{i+1}]")
    s = np.asarray(s, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    psi1 = np.asarray(psi1, dtype=np.float64)
    psi2 = np.asarray(psi2, dtype=np.float64)
    f = pm.pm_force(s, p.np_side, p.nmesh, c["force_scale"]) if force is None else force(s, c["force_scale"])
    v = v + c["kick"] * (f - (c["c1"] * psi1 + c["c2"] * psi2))
    om = p.omega_m
    if c["drift"] == 0.0 and c["dd1"] == 0.0:   # the last step does not drift
        drift = 0.0
    else:
        drift = cosmology.drift_factor(a_i, a_snap, c["a_hi"], om, p.nlpt, p.drift_ansatz)
    s = (s + drift * v + (cosmology.d1(a_snap, om) - cosmology.d1(a_i, om)) * psi1
         + (cosmology.d2(a_snap, om) - cosmology.d2(a_i, om)) * psi2)
    return s, final_velocity(v, psi1, psi2, p, a_snap)


def final_velocity(v_res, psi1, psi2, p: cosmology.Params, a: float = 1.0):
    """Canonical velocity v = v_res + a^2 dx_2LPT/dt at a (H0 = 1, lengths in PM cells; the paper's output velocities, §2.2 eq. motion)."""
    f1, f2 = cosmology.lpt_velocity_factors(a, p.omega_m)
    return v_res + f1 * psi1 + f2 * psi2


def run(white_noise, p: cosmology.Params, nbins: int = 64, steps: int | None = None):
    """A whole realisation: 2LPT IC, n_step COLA steps, P(k) of the final density.

    Returns a dict with psi1, psi2, s, v_res, v (canonical) and pk = (k_mean, P, n_modes).
    ``steps`` stops early (for tests); the default runs all n_step steps.
    """
    psi1, psi2 = lpt.displacements(white_noise, p)
    s, v = initial_state(psi1, psi2, p)
    last = p.nstep if steps is None else steps
    for i in range(1, last + 1):
        s, v = step(i, s, v, psi1, psi2, p)
    out = dict(psi1=psi1, psi2=psi2, s=s, v_res=v)
    out["v"] = final_velocity(v, psi1, psi2, p)
    delta = pm.density_fixed(s, p.np_side, p.nmesh)
    out["pk"] = power.power_spectrum(delta, p.box, nbins)
    return out
