"""GPU parity of every step of the COLA hot path against the FP64 oracle, through the C ABI.

Bars (written per test): integer work (fixed-point deposit, mode counts) is bit-exact; floating
point within the stated FP32 tolerances; whole runs within 1e-3 mesh cells RMS of the final
positions and 0.1% of P(k) for k <= k_Nyq/2 on the 32^3 / 64^3 workload.
"""

import numpy as np
import pytest

import cola_inputs
import oracle
from oracle import cic, cola, cosmology, fourier, lpt, pm, power

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = dict(box=256.0, np_side=32, nmesh=64)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1507_05329_gb300 import build
    build.build()


def ctx_for(**kw):
    from paper_1507_05329_gb300 import Context, Params
    return Context(Params(**kw))


def oparams(**kw):
    return oracle.Params(**kw)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---- S1 deposit: bit-exact ----------------------------------------------------------------
@pytest.mark.parametrize("npd,nm,amp", [(16, 32, 0.0), (16, 32, 3.0), (16, 32, 40.0), (24, 48, 5.0),
                                        (20, 40, 2.5), (32, 48, 7.0), (8, 8, 1.3)])
def test_deposit_bit_exact(npd, nm, amp):
    s = cola_inputs.random_displacements(npd, seed=npd + nm, amplitude=amp)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=100.0)
    rho = ctx.deposit(dev(s))
    ctx.sync()
    got = rho.cpu().numpy().view(np.uint64)
    ref = cic.cic_fixed_mesh(s, npd, nm)
    assert np.array_equal(got, ref)
    assert int(got.sum(dtype=np.uint64)) == npd ** 3 * cic.PARTICLE_MASS


def test_deposit_is_deterministic():
    s = dev(cola_inputs.random_displacements(32, seed=3, amplitude=0.3))   # many particles share cells
    ctx = ctx_for(np_side=32, nmesh=32, box=100.0)
    a = ctx.deposit(s).cpu()
    b = ctx.deposit(s).cpu()
    assert torch.equal(a, b)


# ---- S2 forward FFT of delta ------------------------------------------------------------------
@pytest.mark.parametrize("npd,nm", [(16, 32), (24, 48), (20, 40), (30, 60), (32, 64), (48, 96), (40, 80), (6, 6),
                                    (96, 96)])
def test_density_spectrum(npd, nm):
    s = cola_inputs.random_displacements(npd, seed=nm, amplitude=2.0)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=100.0)
    dk = ctx.density_spectrum(dev(s))
    ctx.sync()
    got = dk.cpu().numpy().astype(np.float64)
    got = got[..., 0] + 1j * got[..., 1]
    ref = fourier.rfft3(pm.density_fixed(s, npd, nm))
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err


# ---- S1-S3 force at particles -----------------------------------------------------------------
@pytest.mark.parametrize("npd,nm,a", [(16, 32, 0.3), (32, 64, 1.0), (24, 48, 0.5), (20, 40, 0.7),
                                      (32, 32, 0.6), (48, 48, 0.9), (64, 64, 0.4), (48, 96, 0.8), (96, 96, 0.5),
                                      (6, 6, 0.7)])
def test_pm_force(npd, nm, a):
    # r = 1 cases are dense enough to take the tile-wise gather from shared memory
    s = cola_inputs.random_displacements(npd, seed=7 * nm, amplitude=1.5)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=100.0)
    f = ctx.pm_force(dev(s), a)
    ctx.sync()
    ref = pm.pm_force(s, npd, nm, 1.5 * 0.27 / a)
    err = np.abs(f.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
    # momentum conservation at any size: the forces sum to zero up to FP32 rounding
    tot = np.abs(f.cpu().numpy().astype(np.float64).sum(axis=1)).max()
    assert tot < 1e-5 * np.abs(ref).sum()


# ---- S0 2LPT ---------------------------------------------------------------------------------
@pytest.mark.parametrize("npd,nm,box", [(16, 32, 128.0), (32, 64, 256.0), (24, 48, 200.0), (20, 40, 150.0),
                                        (96, 96, 300.0), (6, 12, 60.0)])
def test_ic_2lpt(npd, nm, box):
    wn = cola_inputs.white_noise(npd, seed=npd)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=box)
    s, v, psi1, psi2 = ctx.ic_2lpt(dev(wn))
    ctx.sync()
    op = oparams(np_side=npd, nmesh=nm, box=box)
    r1, r2 = lpt.displacements(wn, op)
    e1 = np.abs(psi1.cpu().numpy() - r1).max() / np.abs(r1).max()
    e2 = np.abs(psi2.cpu().numpy() - r2).max() / np.abs(r2).max()
    assert e1 < 2e-6 and e2 < 2e-5, (e1, e2)
    s0, _ = cola.initial_state(r1, r2, op)
    assert np.abs(s.cpu().numpy() - s0).max() < 1e-5 * np.abs(s0).max() + 1e-7
    assert torch.count_nonzero(v) == 0


# ---- S1-S5 one step on identical float32 inputs --------------------------------------------
@pytest.mark.parametrize("i,sched", [(1, None), (5, None), (10, None), (5, 7), (5, 23), (10, 23)])
def test_single_step(i, sched):
    """One step against the oracle, under the default schedule and with the tile-wise kick-drift
    gather (7: one CTA per tile; 23: persistent CTAs staging the next tile meanwhile)."""
    npd, nm = 32, 64
    wn = cola_inputs.white_noise(npd, seed=1)
    op = oparams(**SMALL)
    r1, r2 = lpt.displacements(wn, op)
    rng = np.random.default_rng(i)
    s = (r1 * cosmology.d1(i / 10, 0.27) + rng.normal(0, 0.3, r1.shape)).astype(np.float32)
    v = rng.normal(0, 0.05, r1.shape).astype(np.float32)
    p1, p2 = r1.astype(np.float32), r2.astype(np.float32)
    ctx = ctx_for(**SMALL)
    if sched is not None:
        ctx.schedule = sched
    sg, vg = dev(s), dev(v)
    ctx.step(i, sg, vg, dev(p1), dev(p2))
    ctx.sync()
    rs, rv = cola.step(i, s, v, p1, p2, op)
    assert np.abs(sg.cpu().numpy() - rs).max() < 2e-5 * max(1.0, np.abs(rs).max())
    assert np.abs(vg.cpu().numpy() - rv).max() < 2e-5 * np.abs(rv).max()


# ---- S6 power spectrum on identical positions ---------------------------------------------------
@pytest.mark.parametrize("npd,nm,nb", [(32, 64, 64), (24, 48, 16), (16, 32, 128)])
def test_power_spectrum(npd, nm, nb):
    s = cola_inputs.random_displacements(npd, seed=5, amplitude=2.0)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=300.0)
    pk = ctx.power_spectrum(dev(s), nb)
    ctx.sync()
    k, p, cnt = power.power_spectrum(pm.density_fixed(s, npd, nm), 300.0, nb)
    got = pk.cpu().numpy()
    assert np.array_equal(got[2].astype(np.int64), cnt)
    m = cnt > 0
    np.testing.assert_allclose(got[0][m], k[m], rtol=1e-12)
    np.testing.assert_allclose(got[1][m], p[m], rtol=2e-5)


# ---- whole realisation: the 32^3 / 64^3 workload, 10 steps ------------------------------------
@pytest.fixture(scope="module")
def small_run():
    wn = cola_inputs.white_noise(32, seed=1)
    ctx = ctx_for(**SMALL)
    out = ctx.run(dev(wn), nbins=64)
    ctx.sync()
    ref = cola.run(wn, oparams(**SMALL), nbins=64)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}, ref


def test_run_final_positions_rms(small_run):
    got, ref = small_run
    rms = float(np.sqrt(np.mean((got["s"] - ref["s"]) ** 2)))
    assert rms < 1e-3, rms
    vrms = float(np.sqrt(np.mean((got["v"] - ref["v_res"]) ** 2)) / np.sqrt(np.mean(ref["v_res"] ** 2)))
    assert vrms < 1e-3, vrms


def test_run_power_spectrum(small_run):
    got, ref = small_run
    k, p, cnt = ref["pk"]
    pk = got["pk"]
    assert np.array_equal(pk[2].astype(np.int64), cnt)
    knyq = np.pi * 64 / 256.0
    m = (cnt > 0) & (k <= knyq / 2)
    rel = np.abs(pk[1][m] / p[m] - 1.0)
    assert rel.max() < 1e-3, rel.max()


def test_run_is_bit_reproducible():
    wn = dev(cola_inputs.white_noise(32, seed=1))
    ctx = ctx_for(**SMALL)
    a = ctx.run(wn, nbins=64)
    b = ctx.run(wn, nbins=64)
    ctx.sync()
    for key in ("s", "v", "pk"):
        assert torch.equal(a[key], b[key]), key


def test_run_kernel_count_counts_without_running():
    """cola_run_kernel_count captures one cola_run, counts its kernels and leaves every buffer as it was."""
    from paper_1507_05329_gb300 import ColaError
    wn = dev(cola_inputs.white_noise(32, seed=1))
    ctx = ctx_for(**SMALL)
    out = ctx.run(wn, nbins=64)
    ctx.sync()
    before = {k: out[k].clone() for k in ("s", "v", "psi1", "psi2", "pk")}
    k1 = ctx.run_kernel_count(wn, 64, out=out)
    k2 = ctx.run_kernel_count(wn, 64, out=out)
    ctx.sync()
    assert k1 == k2 and k1 > 10 * 8, (k1, k2)   # at least eight kernels per COLA step
    for key, val in before.items():
        assert torch.equal(val, out[key]), key
    with pytest.raises(ColaError):
        ctx.run_kernel_count(wn, 32, out=dict(out, pk=torch.empty((3, 32), dtype=torch.float64, device="cuda")))


@pytest.mark.parametrize("npd,nm,pipelined", [(32, 64, False), (32, 32, False), (24, 48, False), (32, 64, True),
                                               (24, 48, True)])
def test_run_equals_a_loop_of_steps(npd, nm, pipelined):
    """cola_run is bit-identical to cola_ic_2lpt, separate cola_step calls and cola_power_spectrum,
    with the tile-wise kick-drift gather (one CTA per tile, or persistent CTAs)."""
    from paper_1507_05329_gb300 import binding
    wn = dev(cola_inputs.white_noise(npd, seed=7))
    ctx = ctx_for(np_side=npd, nmesh=nm, box=100.0)
    # the tile-wise gather, selected even where tiles are sparse
    ctx.schedule = (binding.SCHED_BINNED_DEPOSIT | binding.SCHED_TILE_GATHER | binding.SCHED_PIPELINED_FFT
                    | (binding.SCHED_PIPELINED_GATHER if pipelined else 0))
    run = ctx.run(wn, nbins=16)
    s, v, p1, p2 = ctx.ic_2lpt(wn)
    for i in range(1, 11):
        ctx.step(i, s, v, p1, p2)
    pk = ctx.power_spectrum(s, 16)
    ctx.sync()
    assert torch.equal(run["s"], s) and torch.equal(run["v"], v) and torch.equal(run["pk"], pk)


@pytest.mark.parametrize("kw", [dict(ic_mode=1), dict(drift_ansatz=1), dict(nstep=4), dict(nmesh=16)])
def test_run_variants(kw):
    npd = 16
    cfg = dict(box=128.0, np_side=npd, nmesh=32)
    cfg.update(kw)
    wn = cola_inputs.white_noise(npd, seed=9)
    ctx = ctx_for(**cfg)
    out = ctx.run(dev(wn), with_pk=False)
    ctx.sync()
    ref = cola.run(wn, oparams(**cfg), nbins=8)
    rms = float(np.sqrt(np.mean((out["s"].cpu().numpy() - ref["s"]) ** 2)))
    assert rms < 1e-3, rms


# ---- device-side error flags ---------------------------------------------------------------------
def test_nonfinite_state_is_reported():
    from paper_1507_05329_gb300 import ColaError
    npd = 16
    ctx = ctx_for(np_side=npd, nmesh=32, box=100.0)
    s = torch.zeros((3, npd ** 3), device="cuda")
    v = torch.zeros_like(s)
    p1 = torch.zeros_like(s)
    p2 = torch.zeros_like(s)
    p1[0, 5] = float("nan")
    ctx.step(1, s, v, p1, p2)
    with pytest.raises(ColaError) as e:
        ctx.sync()
    assert e.value.status == 5
    ctx.sync()   # the flag is cleared once reported


def test_overflow_is_reported():
    from paper_1507_05329_gb300 import ColaError
    npd, nm = 162, 324   # 162^3 = 4.25e6 > 2^22 particles, all moved onto one mesh node
    ctx = ctx_for(np_side=npd, nmesh=nm, box=100.0)
    q = torch.from_numpy(cic.lattice_indices(npd).astype(np.float32) * 2.0).cuda()
    rho = ctx.deposit(-q)
    with pytest.raises(ColaError) as e:
        ctx.sync()
    assert e.value.status == 4
    del rho


@pytest.mark.parametrize("npd,nm", [(32, 64), (16, 60), (24, 96)])
def test_run_power_spectrum_equals_power_spectrum_of_final_positions(npd, nm):
    """cola_run takes P(k) from the last step's density spectrum (the last step does not drift, so it
    deposits the final positions); that equals cola_power_spectrum of the returned positions: counts and
    mean |k| exactly, P to the FP32 rounding of two FFT kernels.  60 exercises the generic-plan path,
    which recomputes the spectrum instead."""
    from paper_1507_05329_gb300 import Context, Params
    ctx = Context(Params(box=200.0, np_side=npd, nmesh=nm, seed=21))
    out = ctx.run(None, nbins=32)
    again = ctx.power_spectrum(out["s"], 32)
    ctx.sync()
    a, b = out["pk"].cpu().numpy(), again.cpu().numpy()
    assert np.array_equal(a[2], b[2])
    m = b[2] > 0
    np.testing.assert_array_equal(a[0][m], b[0][m])
    np.testing.assert_allclose(a[1][m], b[1][m], rtol=2e-6)
    ctx.close()
