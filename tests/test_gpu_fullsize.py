"""The hot path at the full size the benchmark times (1024^3 particles, 1536^3 mesh, 1200 Mpc/h),
checked where the FP64 oracle cannot run in seconds: against plain PyTorch references of the same
operations (torch.fft, i.e. cuFFT, in FP32; CIC interpolation in FP64 from the same fixed-point
cells and weights), and the 2LPT first order against a torch FP64 restatement with the oracle's
linear power spectrum.  Every schedule the benchmark's autotuner can pick is covered.
"""

import math

import numpy as np
import pytest

import cola_inputs
import oracle
from oracle import cosmology

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NP, NM, BOX = 1024, 1536, 1200.0


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 200 * 2 ** 30:
        pytest.skip("needs about 200 GB of free device memory")
    from paper_1507_05329_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def big():
    from paper_1507_05329_gb300 import Context, Params
    ctx = Context(Params(np_side=NP, nmesh=NM, box=BOX))
    s = cola_inputs.random_displacements_torch(NP, seed=11, amplitude=3.0, device="cuda")
    yield ctx, s
    ctx.close()


def mode_ints(n, half=False):
    m = torch.arange(n // 2 + 1 if half else n, device="cuda", dtype=torch.float64)
    return m if half else torch.where(m < n // 2, m, m - n)


def reference_delta(rho):
    """delta = rho N^3 / (n 2^42) - 1 in FP64, stored FP32 (slab by slab to bound memory)."""
    scale = NM ** 3 / (NP ** 3 * 2.0 ** 42)
    delta = torch.empty((NM, NM, NM), dtype=torch.float32, device="cuda")
    for x0 in range(0, NM, 128):
        delta[x0:x0 + 128] = (rho[x0:x0 + 128].double() * scale - 1.0).float()
    return delta


def fixed_cells(s, ids):
    """Fixed-point cell and 14-bit weight of the sampled particles (the deposit's definition)."""
    r_fixed = (NM << 20) // NP
    q = torch.stack([ids // (NP * NP), (ids // NP) % NP, ids % NP])
    g = q * r_fixed + torch.round(s[:, ids].double() * 2.0 ** 20).long()
    g = torch.remainder(g, NM << 20)
    return g >> 20, ((g >> 6) & 16383).double() / 16384.0


# default (wide tiles, in-place pipelined passes); narrow tiles with: 8-element pipelined passes; + pipelined
# gather; + 8-element Green; + 8-element C2R; + pipelined C2R; 8-element R2C; plain strided passes, narrow and wide;
# in-place pipelined passes; three-buffer pipelined passes with the wide Green pass
SCHEDULES = [None, 15, 31, 47, 79, 143, 1031, 3, 2051, 6151, 2055]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_fullsize_density_spectrum_and_force(big, sched):
    """delta(k) of the GPU path against torch.fft.rfftn of the same deposited mesh (FP32 cuFFT):
    rms difference < 2e-6 of the rms mode, every mode within 1e-3 of it (k = 0 excluded, the GPU
    keeps the mean); the PM force at 2^20 sampled particles against an FP32 cuFFT force mesh and an
    FP64 CIC interpolation: max error < 1e-4 of the largest force."""
    ctx, s = big
    if sched is not None:
        ctx.schedule = sched
    rho = ctx.deposit(s)
    ctx.sync()                                    # the library's exact 128-bit mass check
    delta = reference_delta(rho)
    del rho
    ref = torch.fft.rfftn(delta)
    del delta
    got = torch.view_as_complex(ctx.density_spectrum(s))
    ctx.sync()
    ref[0, 0, 0] = 0
    got[0, 0, 0] = 0
    rms = ref.abs().pow(2).mean().sqrt()
    diff = (got - ref).abs()
    del got
    assert float(diff.pow(2).mean().sqrt() / rms) < 2e-6
    assert float(diff.max() / rms) < 1e-3
    del diff
    # force mesh F_j = irfft(i D(k_j) g(k) delta(k)), g = force_scale / k^2, k = 2 pi m / N (cells)
    a = 0.5
    fs = 1.5 * 0.27 / a
    kf = 2.0 * math.pi / NM
    mx, my, mz = mode_ints(NM), mode_ints(NM), mode_ints(NM, half=True)

    def dker(m):
        k = kf * m
        d = (8.0 * torch.sin(k) - torch.sin(2.0 * k)) / 6.0
        return torch.where(m.abs() * 2 == NM, torch.zeros_like(d), d)

    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    ids = torch.randint(0, NP ** 3, (1 << 20,), generator=gen, device="cuda")
    cell, w1 = fixed_cells(s, ids)
    fgot = ctx.pm_force(s, a)[:, ids].double()
    ctx.sync()
    fref = torch.zeros((3, ids.numel()), dtype=torch.float64, device="cuda")
    k2yz = (kf * my).view(NM, 1) ** 2 + (kf * mz).view(1, NM // 2 + 1) ** 2
    for j in range(3):
        fk = torch.empty_like(ref)
        for x0 in range(0, NM, 128):   # the multiplier slab by slab (FP64), applied in FP32
            k2 = (kf * mx[x0:x0 + 128]).view(-1, 1, 1) ** 2 + k2yz.view(1, NM, NM // 2 + 1)
            g = fs / torch.where(k2 > 0, k2, torch.ones_like(k2))
            g[k2 == 0] = 0.0
            d = (dker(mx[x0:x0 + 128]).view(-1, 1, 1), dker(my).view(1, NM, 1),
                 dker(mz).view(1, 1, NM // 2 + 1))[j]
            fk[x0:x0 + 128] = ref[x0:x0 + 128] * (1j * (d * g).float())
            del k2, g
        fmesh = torch.fft.irfftn(fk, s=(NM, NM, NM))
        del fk
        for dx in (0, 1):
            wx = w1[0] if dx else 1.0 - w1[0]
            ix = (cell[0] + dx) % NM
            for dy in (0, 1):
                wy = w1[1] if dy else 1.0 - w1[1]
                iy = (cell[1] + dy) % NM
                for dz in (0, 1):
                    wz = w1[2] if dz else 1.0 - w1[2]
                    iz = (cell[2] + dz) % NM
                    fref[j] += wx * wy * wz * fmesh[ix, iy, iz].double()
        del fmesh
    del ref
    torch.cuda.empty_cache()
    err = (fgot - fref).abs().max() / fref.abs().max()
    assert float(err) < 1e-4, float(err)


def test_fullsize_2lpt_first_order(big):
    """Psi1 of cola_ic_2lpt at 1024^3 against a torch FP64 restatement: W = rfft(w), Psi1_j =
    irfft(i kodd_j sqrt(P(k)/V_cell) W / k^2) in mesh cells, P from the oracle's sigma8-normalised
    BBKS spectrum on the integer |m|^2 of the lattice.  rms difference < 1e-5 of the rms."""
    ctx, _ = big
    wn = cola_inputs.white_noise_torch(NP, 3, "cuda")
    s, v, psi1, psi2 = ctx.ic_2lpt(wn)
    ctx.sync()
    del s, v, psi2
    op = oracle.Params(box=BOX, np_side=NP, nmesh=NM)
    amp = cosmology.power_amplitude(op)
    m2max = 3 * (NP // 2) ** 2
    kk = 2.0 * np.pi * np.sqrt(np.arange(1, m2max + 1, dtype=np.float64)) / BOX
    table = np.concatenate([[0.0], np.sqrt(cosmology.linear_power(kk, op, amp) / (BOX / NP) ** 3)])
    table = torch.from_numpy(table).cuda()
    wk = torch.fft.rfftn(wn.view(NP, NP, NP).double())
    mx, my, mz = mode_ints(NP), mode_ints(NP), mode_ints(NP, half=True)
    m2 = (mx.view(NP, 1, 1) ** 2 + my.view(1, NP, 1) ** 2 + mz.view(1, 1, NP // 2 + 1) ** 2)
    wk *= table[m2.long()]
    klat = 2.0 * math.pi / NP
    inv = torch.where(m2 > 0, 1.0 / (m2 * klat * klat), torch.zeros_like(m2))
    del m2
    r = NM / NP
    for j, (m, shape) in enumerate(((mx, (NP, 1, 1)), (my, (1, NP, 1)), (mz, (1, 1, NP // 2 + 1)))):
        kodd = torch.where(m.abs() * 2 == NP, torch.zeros_like(m), m) * klat
        ref = torch.fft.irfftn(wk * (1j * kodd.view(shape) * inv), s=(NP, NP, NP)).reshape(-1) * r
        got = psi1[j].double()
        rel = (got - ref).pow(2).mean().sqrt() / ref.pow(2).mean().sqrt()
        assert float(rel) < 1e-5, (j, float(rel))
        del ref, got
