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
