"""GPU parity of the paper's variants against the FP64 oracle: snapshots between steps (§2.2),
snapshot runs at the paper's output redshifts z = 0.73, 0.6, 0.44, 0 (§3), the n_step sweep, and
the CIC smoothing/alias-corrected power spectrum (§3.3, Jing 2005, flat-spectrum form)."""

import numpy as np
import pytest

import cola_inputs
import oracle
from oracle import cola, cosmology, lpt, pm, power

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = dict(box=256.0, np_side=32, nmesh=64)
Z_OUT = (0.73, 0.6, 0.44, 0.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1507_05329_gb300 import build
    build.build()


def ctx_for(**kw):
    from paper_1507_05329_gb300 import Context, Params
    return Context(Params(**kw))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("i,frac", [(3, 0.0), (3, 0.37), (6, 0.81), (9, 1.0), (10, 0.0)])
def test_snapshot_matches_oracle(i, frac):
    """GPU: step i then cola_snapshot back from a_{i+1}; oracle: kick then drift forward to a_snap.
    Same bar as the single-step parity test (2e-5 of the largest value)."""
    npd = 32
    wn = cola_inputs.white_noise(npd, seed=1)
    op = oracle.Params(**SMALL)
    r1, r2 = lpt.displacements(wn, op)
    rng = np.random.default_rng(i)
    s = (r1 * cosmology.d1(i / 10, 0.27) + rng.normal(0, 0.3, r1.shape)).astype(np.float32)
    v = rng.normal(0, 0.05, r1.shape).astype(np.float32)
    p1, p2 = r1.astype(np.float32), r2.astype(np.float32)
    c = cosmology.step_scalars(op, i)
    a_snap = c["a"] + frac * (c["a_next"] - c["a"])
    ctx = ctx_for(**SMALL)
    sg, vg = dev(s), dev(v)
    ctx.step(i, sg, vg, dev(p1), dev(p2))
    so, vo = ctx.snapshot(i, a_snap, sg, vg, dev(p1), dev(p2))
    ctx.sync()
    rs, rv = cola.snapshot(i, s, v, p1, p2, op, a_snap)
    assert np.abs(so.cpu().numpy() - rs).max() < 2e-5 * max(1.0, np.abs(rs).max())
    assert np.abs(vo.cpu().numpy() - rv).max() < 2e-5 * np.abs(rv).max()


def test_snapshot_rejects_times_outside_the_step():
    from paper_1507_05329_gb300 import ColaError
    ctx = ctx_for(**SMALL)
    z = ctx.empty_particles().zero_()
    with pytest.raises(ColaError):
        ctx.snapshot(3, 0.45, z, z, z, z)
    with pytest.raises(ColaError):
        ctx.snapshot(10, 0.99, z, z, z, z)


@pytest.fixture(scope="module")
def snapshot_run():
    a_out = [1.0 / (1.0 + z) for z in Z_OUT]
    wn = cola_inputs.white_noise(32, seed=1)
    ctx = ctx_for(**SMALL)
    got = ctx.run_snapshots(dev(wn), a_out, nbins=64)
    plain = ctx.run(dev(wn), nbins=64)
    ctx.sync()
    got = {k: v.cpu().numpy() for k, v in got.items()}
    plain = {k: v.cpu().numpy() for k, v in plain.items()}
    op = oracle.Params(**SMALL)
    psi1, psi2 = lpt.displacements(wn, op)
    s, v = cola.initial_state(psi1, psi2, op)
    ref = []
    k = 0
    for i in range(1, op.nstep + 1):
        c = cosmology.step_scalars(op, i)
        while k < len(a_out) and a_out[k] <= c["a_next"] + 1e-12:
            ss, vs = cola.snapshot(i, s, v, psi1, psi2, op, a_out[k])
            ref.append((ss, vs, power.power_spectrum(pm.density_fixed(ss.astype(np.float32), 32, 64), 256.0, 64)))
            k += 1
        s, v = cola.step(i, s, v, psi1, psi2, op)
    return got, plain, ref


def test_snapshot_run_positions_and_velocities(snapshot_run):
    """Whole-run bar at every output redshift: positions within 1e-3 cells RMS, velocities 1e-3
    relative RMS."""
    got, _, ref = snapshot_run
    assert len(ref) == len(Z_OUT)
    for k, (rs, rv, _) in enumerate(ref):
        rms = float(np.sqrt(np.mean((got["s_snap"][k] - rs) ** 2)))
        assert rms < 1e-3, (k, rms)
        vrms = float(np.sqrt(np.mean((got["v_snap"][k] - rv) ** 2)) / np.sqrt(np.mean(rv ** 2)))
        assert vrms < 1e-3, (k, vrms)


def test_snapshot_run_power_spectra(snapshot_run):
    """P(k) at every output redshift within 0.1% for k <= k_Nyq / 2, mode counts exact."""
    got, _, ref = snapshot_run
    knyq = np.pi * 64 / 256.0
    for k, (_, _, (kk, p, cnt)) in enumerate(ref):
        pk = got["pk_snap"][k]
        assert np.array_equal(pk[2].astype(np.int64), cnt)
        m = (cnt > 0) & (kk <= knyq / 2)
        rel = np.abs(pk[1][m] / p[m] - 1.0)
        assert rel.max() < 1e-3, (k, rel.max())


def test_snapshot_run_ends_like_a_plain_run(snapshot_run):
    """The a = 1 snapshot is the final state (bit-identical positions; canonical velocity), and the
    run's own outputs equal cola_run's."""
    got, plain, _ = snapshot_run
    assert np.array_equal(got["s"], plain["s"]) and np.array_equal(got["v"], plain["v"])
    assert np.array_equal(got["s_snap"][-1], plain["s"])
    assert np.array_equal(got["pk_snap"][-1], plain["pk"])


@pytest.mark.parametrize("nstep", [20, 50, 100])
def test_nstep_sweep(nstep):
    """The paper's step-count study: a 16^3 / 32^3 run with 20 and 50 COLA steps against the oracle,
    final positions within 1e-3 cells RMS."""
    cfg = dict(box=128.0, np_side=16, nmesh=32, nstep=nstep)
    wn = cola_inputs.white_noise(16, seed=9)
    ctx = ctx_for(**cfg)
    out = ctx.run(dev(wn), with_pk=False)
    ctx.sync()
    ref = cola.run(wn, oracle.Params(**cfg), nbins=8)
    rms = float(np.sqrt(np.mean((out["s"].cpu().numpy() - ref["s"]) ** 2)))
    assert rms < 1e-3, rms


@pytest.mark.parametrize("npd,nm,amp", [(32, 64, 2.0), (24, 48, 0.5), (16, 32, 6.0)])
def test_cic_corrected_power_spectrum(npd, nm, amp):
    """Corrected P(k) on identical positions: each mode's P_raw / C2 - V/n in FP64 from the FP32
    spectrum; bar 1e-4 of (|P| + V/n) per bin, mode counts exact, uncorrected output unchanged."""
    s = cola_inputs.random_displacements(npd, seed=npd + 1, amplitude=amp)
    ctx = ctx_for(np_side=npd, nmesh=nm, box=300.0)
    got = ctx.power_spectrum_ex(dev(s), 32, cic_correct=True).cpu().numpy()
    raw = ctx.power_spectrum_ex(dev(s), 32, cic_correct=False).cpu().numpy()
    plain = ctx.power_spectrum(dev(s), 32).cpu().numpy()
    ctx.sync()
    assert np.array_equal(raw, plain)
    delta = pm.density_fixed(s, npd, nm)
    k, p, cnt = power.power_spectrum(delta, 300.0, 32, cic_correct=True, n_particles=npd ** 3)
    assert np.array_equal(got[2].astype(np.int64), cnt)
    shot = 300.0 ** 3 / npd ** 3
    m = cnt > 0
    assert np.all(np.abs(got[1][m] - p[m]) <= 1e-4 * (np.abs(p[m]) + shot))
