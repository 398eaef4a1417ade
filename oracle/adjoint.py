"""Oracle: the differentiable COLA model and its hand-written adjoint (reverse mode) in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

The paper has no adjoint; this is the transpose of the forward model of ``cola.py`` (§2.1, §2.2
eqs. cola-kick and cola-drift, PM force of §2.2/§2.3, 2LPT of §2.1/§2.3) with one change that
differentiation needs: the CIC weights are the continuous ones (``cic_exact_mesh`` and exact
interpolation weights), since the fixed-point weights are piecewise constant in position (their
derivative is zero almost everywhere).  The derivative of a CIC weight is taken one-sided at cell
faces, from the cell floor(x) chooses (a reading: the paper has no adjoint).

Loss (the differentiable workload): L = sum_g (delta_g - delta_target_g)^2 over a CIC density
contrast on an ngrid^3 grid of the final positions.

Linear maps are transposed with the rule: for y -> irfftn(M rfftn(y)) with a Hermitian multiplier
M (M(-k) = conj M(k)), the transpose is y -> irfftn(conj(M) rfftn(y)) (same normalisation).
"""

from __future__ import annotations

import numpy as np

from . import cic, cosmology, fourier, lpt, pm


# ---- continuous CIC pieces ------------------------------------------------------------------
def _positions(s, np_side: int, nmesh: int) -> np.ndarray:
    """Mesh coordinates x = q r + s (PM cells), not wrapped."""
    return cic.lattice_indices(np_side) * (nmesh / np_side) + np.asarray(s, dtype=np.float64)


def _cells(x, n: int):
    xm = np.mod(x, n)
    c = np.floor(xm).astype(np.int64)
    return c, xm - c


def interp_exact(fields, x, n: int) -> np.ndarray:
    """CIC interpolation of fields [m, n, n, n] at positions x [3, p] (continuous weights)."""
    c, t = _cells(x, n)
    return cic.cic_interp(fields, c, t)


def interp_grad_exact(field, x, n: int) -> np.ndarray:
    """Gradient [3, p] of the CIC interpolant of one field [n, n, n] at x: dW/dx_d = +-1 times the
    other two axes' weights."""
    c, t = _cells(x, n)
    f = np.asarray(field, dtype=np.float64)
    out = np.zeros((3, x.shape[1]))
    for dx in (0, 1):
        wx, gx = (t[0], 1.0) if dx else (1.0 - t[0], -1.0)
        ix = (c[0] + dx) % n
        for dy in (0, 1):
            wy, gy = (t[1], 1.0) if dy else (1.0 - t[1], -1.0)
            iy = (c[1] + dy) % n
            for dz in (0, 1):
                wz, gz = (t[2], 1.0) if dz else (1.0 - t[2], -1.0)
                iz = (c[2] + dz) % n
                v = f[ix, iy, iz]
                out[0] += gx * wy * wz * v
                out[1] += wx * gy * wz * v
                out[2] += wx * wy * gz * v
    return out


def deposit_exact(values, x, n: int) -> np.ndarray:
    """CIC deposit of per-particle values [m, p] onto m meshes [m, n, n, n] (continuous weights)."""
    c, t = _cells(x, n)
    values = np.atleast_2d(np.asarray(values, dtype=np.float64))
    out = np.zeros((values.shape[0], n ** 3))
    for dx in (0, 1):
        wx = t[0] if dx else 1.0 - t[0]
        ix = (c[0] + dx) % n
        for dy in (0, 1):
            wy = t[1] if dy else 1.0 - t[1]
            iy = (c[1] + dy) % n
            for dz in (0, 1):
                wz = t[2] if dz else 1.0 - t[2]
                idx = (ix * n + iy) * n + (c[2] + dz) % n
                w = wx * wy * wz
                for m in range(values.shape[0]):
                    np.add.at(out[m], idx, w * values[m])
    return out.reshape((values.shape[0], n, n, n))


# ---- differentiable forward --------------------------------------------------------------------
def pm_force_exact(s, np_side: int, nmesh: int, force_scale: float) -> np.ndarray:
    """PM force [3, n] with continuous CIC weights (same Green/gradient kernels as ``pm``)."""
    x = _positions(s, np_side, nmesh)
    rho = deposit_exact(np.ones((1, x.shape[1])), x, nmesh)[0]
    delta = rho * (nmesh ** 3 / x.shape[1]) - 1.0
    return interp_exact(pm.force_mesh(delta, force_scale), x, nmesh)


def grid_delta(s, np_side: int, nmesh: int, ngrid: int) -> np.ndarray:
    """Density contrast of the particles on an ngrid^3 CIC grid (grid coordinate x ngrid/nmesh)."""
    y = _positions(s, np_side, nmesh) * (ngrid / nmesh)
    rho = deposit_exact(np.ones((1, y.shape[1])), y, ngrid)[0]
    return rho * (ngrid ** 3 / y.shape[1]) - 1.0


def forward(white_noise, p: cosmology.Params, checkpoints: bool = False):
    """2LPT + n_step COLA steps with the continuous-CIC force.  Returns psi1, psi2, s (final) and,
    with checkpoints, the list of positions s_i at which step i evaluated its force."""
    from . import cola
    psi1, psi2 = lpt.displacements(white_noise, p)
    s, v = cola.initial_state(psi1, psi2, p)
    ck = []
    for i in range(1, p.nstep + 1):
        if checkpoints:
            ck.append(s.copy())
        s, v = cola.step(i, s, v, psi1, psi2, p,
                         force=lambda ss, fs: pm_force_exact(ss, p.np_side, p.nmesh, fs))
    return dict(psi1=psi1, psi2=psi2, s=s, v=v, checkpoints=ck)


def loss(white_noise, p: cosmology.Params, ngrid: int, target) -> float:
    d = grid_delta(forward(white_noise, p)["s"], p.np_side, p.nmesh, ngrid)
    return float(np.sum((d - target) ** 2))


# ---- adjoints ------------------------------------------------------------------------------------
def grid_delta_adjoint(s, np_side: int, nmesh: int, ngrid: int, lam_delta) -> np.ndarray:
    """d/ds of sum_g lam_delta_g delta_g(s): [3, n]."""
    y = _positions(s, np_side, nmesh) * (ngrid / nmesh)
    g = interp_grad_exact(lam_delta, y, ngrid) * (ngrid ** 3 / y.shape[1])
    return g * (ngrid / nmesh)


def pm_force_adjoint(s, lam_f, np_side: int, nmesh: int, force_scale: float) -> np.ndarray:
    """d/ds of sum_p lam_f_p . F_p(s) for the continuous-CIC PM force: [3, n].

    Interpolation term: grad W(x_p - c) . (lam_f_p . F_c).  Density term: the 3 meshes
    deposit(lam_f_j) go through the transposed Green/gradient multipliers conj(i D(k_j) g(k)) into one
    mesh lam_delta, lam_rho = lam_delta N^3/n, gathered with grad W."""
    x = _positions(s, np_side, nmesh)
    n = x.shape[1]
    nm = nmesh
    rho = deposit_exact(np.ones((1, n)), x, nm)[0]
    delta = rho * (nm ** 3 / n) - 1.0
    fmesh = pm.force_mesh(delta, force_scale)
    lam_f = np.asarray(lam_f, dtype=np.float64)
    out = np.zeros((3, n))
    for j in range(3):   # interpolation term: F_j interpolant gradient times lam_f_j
        out += interp_grad_exact(fmesh[j], x, nm) * lam_f[j]
    lam_meshes = deposit_exact(lam_f, x, nm)
    mx, my, mz = fourier.mode_grids(nm)
    kf = 2.0 * np.pi / nm
    k2 = (mx * mx + my * my + mz * mz).astype(np.float64) * kf * kf
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(k2 > 0, force_scale / k2, 0.0)
    lam_dk = np.zeros(k2.shape[:2] + (nm // 2 + 1,), dtype=np.complex128)
    for j, m in enumerate((mx, my, mz)):
        mult = 1j * pm.gradient_kernel(m, nm) * g
        lam_dk = lam_dk + np.conj(mult) * fourier.rfft3(lam_meshes[j])
    lam_delta = fourier.irfft3(lam_dk, nm)
    out += interp_grad_exact(lam_delta * (nm ** 3 / n), x, nm)
    return out


def lpt_adjoint(white_noise, lam_psi1, lam_psi2, p: cosmology.Params) -> np.ndarray:
    """d/dw of sum (lam_psi1 . Psi1(w) + lam_psi2 . Psi2(w)) for the 2LPT maps of ``lpt``: [n]."""
    npd = p.np_side
    dk = lpt.linear_density_k(white_noise, p)
    # amplitude sqrt(P(k)/V_cell) as a multiplier: delta_L(k) = amp W(k)
    mx, my, mz = fourier.mode_grids(npd)
    kf = 2.0 * np.pi / p.box
    kmag = np.sqrt((mx * mx + my * my + mz * mz).astype(np.float64)) * kf
    a = cosmology.power_amplitude(p)
    pk = np.where(kmag > 0, cosmology.linear_power(np.where(kmag > 0, kmag, 1.0), p, a), 0.0)
    amp = np.sqrt(pk / (p.box / npd) ** 3)
    k_full = [m.astype(np.float64) * kf for m in (mx, my, mz)]
    k_odd = [fourier.odd_mode(m, npd).astype(np.float64) * kf for m in (mx, my, mz)]
    k2 = k_full[0] ** 2 + k_full[1] ** 2 + k_full[2] ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_k2 = np.where(k2 > 0, 1.0 / k2, 0.0)
    to_cells = p.nmesh / p.box
    lam1 = np.asarray(lam_psi1, dtype=np.float64).reshape(3, npd, npd, npd) * to_cells
    lam2 = np.asarray(lam_psi2, dtype=np.float64).reshape(3, npd, npd, npd) * to_cells
    # first order: Psi1_j = irfft(i kodd_j inv_k2 amp W)
    acc = np.zeros_like(dk)
    for j in range(3):
        acc = acc + np.conj(1j * k_odd[j] * inv_k2 * amp) * fourier.rfft3(lam1[j])
    # second order: Psi2_j = irfft(-i kodd_j inv_k2 rfft(S)), S = sum_{a<b} phi_aa phi_bb - phi_ab^2
    lam_s = np.zeros((npd, npd, npd))
    for j in range(3):
        lam_s += fourier.irfft3(np.conj(-1j * k_odd[j] * inv_k2) * fourier.rfft3(lam2[j]), npd)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    hmult = {}
    phi = {}
    for (i, j) in pairs:
        kk = k_full[i] * k_full[i] if i == j else k_odd[i] * k_odd[j]
        hmult[(i, j)] = kk * inv_k2
        phi[(i, j)] = fourier.irfft3(hmult[(i, j)] * dk, npd)
    dS = {(0, 0): phi[(1, 1)] + phi[(2, 2)], (1, 1): phi[(0, 0)] + phi[(2, 2)],
          (2, 2): phi[(0, 0)] + phi[(1, 1)], (0, 1): -2.0 * phi[(0, 1)],
          (0, 2): -2.0 * phi[(0, 2)], (1, 2): -2.0 * phi[(1, 2)]}
    for key in pairs:
        acc = acc + np.conj(hmult[key] * amp) * fourier.rfft3(lam_s * dS[key])
    return fourier.irfft3(acc, npd).ravel()


def gradient(white_noise, p: cosmology.Params, ngrid: int, target):
    """(L, dL/dw) of the differentiable workload, by the hand-written adjoint."""
    fwd = forward(white_noise, p, checkpoints=True)
    psi1, psi2 = fwd["psi1"], fwd["psi2"]
    d = grid_delta(fwd["s"], p.np_side, p.nmesh, ngrid)
    lval = float(np.sum((d - target) ** 2))
    lam_s = grid_delta_adjoint(fwd["s"], p.np_side, p.nmesh, ngrid, 2.0 * (d - target))
    lam_v = np.zeros_like(lam_s)
    lam_p1 = np.zeros_like(lam_s)
    lam_p2 = np.zeros_like(lam_s)
    for i in range(p.nstep, 0, -1):
        c = cosmology.step_scalars(p, i)
        # s_{i+1} = s_i + drift v + dd1 Psi1 + dd2 Psi2
        lam_v = lam_v + c["drift"] * lam_s
        lam_p1 = lam_p1 + c["dd1"] * lam_s
        lam_p2 = lam_p2 + c["dd2"] * lam_s
        # v_{i+1/2} = v_{i-1/2} + kick (F(s_i) - c1 Psi1 - c2 Psi2)
        lam_f = c["kick"] * lam_v
        lam_p1 = lam_p1 - c["c1"] * lam_f
        lam_p2 = lam_p2 - c["c2"] * lam_f
        lam_s = lam_s + pm_force_adjoint(fwd["checkpoints"][i - 1], lam_f, p.np_side, p.nmesh,
                                         c["force_scale"])
    a1 = 1.0 / p.nstep
    lam_p1 = lam_p1 + cosmology.d1(a1, p.omega_m) * lam_s
    lam_p2 = lam_p2 + cosmology.d2(a1, p.omega_m) * lam_s
    return lval, lpt_adjoint(white_noise, lam_p1, lam_p2, p)
