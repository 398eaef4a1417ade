"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle's callers.

This module holds no arithmetic of the COLA method: it only draws random numbers and builds
the workload descriptions.  Both the CUDA path and the oracle receive what it returns as inputs.

Workloads (periodic boxes, flat LCDM Om=0.27, h=0.7, ns=0.96, sigma8=0.8, BBKS P(k), 10 steps):
  * small     : L=256 Mpc/h,  32^3 particles,   64^3 mesh, seed 1
  * medium    : L=600 Mpc/h, 256^3 particles,  512^3 mesh, seed 2
  * large     : L=1200 Mpc/h, 1024^3 particles, 1536^3 mesh, seed 3
  * adjoint   : L=400 Mpc/h, 128^3 particles,  256^3 mesh, seed 4 (target from seed 5)
  * batched   : 24 x (300 Mpc/h, 96^3, 192^3), 24 x (400, 128^3, 256^3), 16 x (500, 160^3, 320^3),
                seeds 100..163
"""

from __future__ import annotations

import numpy as np

COSMOLOGY = dict(omega_m=0.27, h=0.7, n_s=0.96, sigma8=0.8)

WORKLOADS = {
    "small": dict(box=256.0, np_side=32, nmesh=64, seed=1),
    "medium": dict(box=600.0, np_side=256, nmesh=512, seed=2),
    "large": dict(box=1200.0, np_side=1024, nmesh=1536, seed=3),
    "adjoint": dict(box=400.0, np_side=128, nmesh=256, seed=4),
}


# loss of the differentiable workload: CIC grid of the final density, target realisation, and the
# central finite-difference check (step, number of directions, largest |m| of a direction)
ADJOINT_LOSS = dict(ngrid=64, target_seed=5, fd_eps=1e-3, fd_modes=32, fd_mmax=6)


def batched_workload():
    """The 64 uneven realisations of the batched-mock workload as a list of dicts."""
    out = []
    seed = 100
    for count, box, npd, nm in ((24, 300.0, 96, 192), (24, 400.0, 128, 256), (16, 500.0, 160, 320)):
        for _ in range(count):
            out.append(dict(box=box, np_side=npd, nmesh=nm, seed=seed))
            seed += 1
    return out


def white_noise(np_side: int, seed: int) -> np.ndarray:
    """Unit Gaussian white noise, one float32 per lattice site, flat index (ix*Np+iy)*Np+iz."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(np_side ** 3, dtype=np.float32)


def random_displacements(np_side: int, seed: int, amplitude: float) -> np.ndarray:
    """float32 [3, n] displacements (mesh cells), Gaussian with the given rms per axis."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((3, np_side ** 3)) * amplitude).astype(np.float32)


def random_field(shape, seed: int) -> np.ndarray:
    """float32 unit Gaussian array of the given shape."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape).astype(np.float32)


def white_noise_torch(np_side: int, seed: int, device):
    """Unit Gaussian white noise drawn on the device by torch's seeded generator (large workloads,
    where drawing 10^9 values on the host would dominate the set-up time)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn(np_side ** 3, generator=g, device=device, dtype=torch.float32)


def plane_wave_directions(np_side: int, count: int, seed: int, mmax: int) -> np.ndarray:
    """float32 [count, np^3] real plane waves cos(2 pi m.q / np + phase) of unit amplitude per
    lattice site (the white noise's own per-site scale), m a random nonzero integer vector with
    |m_i| <= mmax, phase uniform in [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    q = np.arange(np_side, dtype=np.float64)
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    out = np.empty((count, np_side ** 3), dtype=np.float32)
    for i in range(count):
        m = np.zeros(3, dtype=np.int64)
        while not m.any():
            m = rng.integers(-mmax, mmax + 1, size=3)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        out[i] = np.cos(2.0 * np.pi * (m[0] * qx + m[1] * qy + m[2] * qz) / np_side + ph).ravel()
    return out


def random_displacements_torch(np_side: int, seed: int, amplitude: float, device):
    """float32 [3, n] Gaussian displacements (mesh cells) drawn on the device by torch's seeded
    generator (full-size tests, where drawing 3 x 10^9 values on the host is slow)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn((3, np_side ** 3), generator=g, device=device, dtype=torch.float32) * amplitude
