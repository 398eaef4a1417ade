"""Execution schedules, the autotuner and batched realisations in one CUDA graph, on the GPU.

Every schedule runs the same method (§2.2, §2.3): the fixed-point deposit must stay bit-exact
against the oracle under every schedule, and the PM force must agree with the oracle to the
tolerance of the single-realisation parity tests.  A batch is a set of independent cola_run calls
(the paper's mock catalogues, §3): each member's results must equal a plain single-context run
bit for bit, eagerly and from the replayed graph.
"""

import numpy as np
import pytest

import cola_inputs
import oracle
from oracle import cic, cola, pm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1507_05329_gb300 import build
    build.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def all_schedules(ctx):
    """Every valid combination of the knobs below the budget bits, then each of those with the R2C
    and tile-width knobs flipped together, and with the in-place pipelined passes where valid."""
    from paper_1507_05329_gb300 import binding as b
    low = [sc for sc in range(4 << b.SCHED_BUDGET_SHIFT) if ctx._schedule_ok(sc)]
    both = b.SCHED_R2C_EPT8 | b.SCHED_WIDE_TILES
    extra = [sc | both for sc in low] + [sc | b.SCHED_PIPE_INPLACE for sc in low
                                         if ctx._schedule_ok(sc | b.SCHED_PIPE_INPLACE)]
    assert all(ctx._schedule_ok(sc) for sc in extra)
    return low + extra


# ---- schedules -----------------------------------------------------------------------------
@pytest.mark.parametrize("npd,nm,amp", [(32, 64, 4.0), (48, 96, 2.0), (24, 72, 6.0)])
def test_every_schedule_deposits_bit_exactly(npd, nm, amp):
    from paper_1507_05329_gb300 import Context, Params
    s = cola_inputs.random_displacements(npd, seed=npd + 7, amplitude=amp)
    ctx = Context(Params(np_side=npd, nmesh=nm, box=100.0))
    ref = cic.cic_fixed_mesh(s, npd, nm)
    scheds = all_schedules(ctx)
    assert len(scheds) >= 2
    for sc in scheds:
        ctx.schedule = sc
        assert ctx.schedule == sc
        got = ctx.deposit(dev(s)).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, ref), sc
    ctx.sync()


@pytest.mark.parametrize("npd,nm", [(32, 64), (24, 72), (48, 192)])   # 192 = 8 8 3: a middle stage
def test_every_schedule_gives_the_oracle_force(npd, nm):
    """Same bar as the single-schedule force parity: max error < 1e-5 of the largest force."""
    from paper_1507_05329_gb300 import Context, Params
    s = cola_inputs.random_displacements(npd, seed=3 * npd, amplitude=1.5)
    a = 0.5
    ref = pm.pm_force(s, npd, nm, 1.5 * 0.27 / a)
    ctx = Context(Params(np_side=npd, nmesh=nm, box=100.0))
    for sc in all_schedules(ctx):
        ctx.schedule = sc
        f = ctx.pm_force(dev(s), a).cpu().numpy()
        err = np.abs(f - ref).max() / np.abs(ref).max()
        assert err < 1e-5, (sc, err)
    ctx.sync()


def test_invalid_schedules_are_rejected():
    from paper_1507_05329_gb300 import ColaError, Context, Params, binding
    ctx = Context(Params(np_side=32, nmesh=64, box=100.0))
    for bad in (binding.SCHED_TILE_GATHER, 1 << 13, 3 << binding.SCHED_BUDGET_SHIFT,
                1 << binding.SCHED_BUDGET_SHIFT,   # budget without the pipelined passes
                binding.SCHED_PIPE_INPLACE,        # in place without the pipelined passes
                binding.SCHED_PIPE_INPLACE | binding.SCHED_PIPELINED_FFT | (1 << binding.SCHED_BUDGET_SHIFT),
                binding.SCHED_PIPE_INPLACE | binding.SCHED_PIPELINED_FFT | binding.SCHED_PIPE_EPT8):
        with pytest.raises(ColaError):
            ctx.schedule = bad


def test_autotune_keeps_the_fastest_valid_schedule():
    from paper_1507_05329_gb300 import Context, Params
    ctx = Context(Params(np_side=32, nmesh=64, box=100.0))
    w = dev(cola_inputs.white_noise(32, seed=1))
    out = ctx.run(w, with_pk=False)
    best, times = ctx.autotune(out["s"], reps=2)
    assert best in times and best == ctx.schedule
    assert all(t > 0 for t in times.values())
    assert times[best] == min(times.values())
    # the tuned context still runs the method exactly as before (deposit is schedule independent)
    rho = ctx.deposit(out["s"]).cpu().numpy().view(np.uint64)
    assert np.array_equal(rho, cic.cic_fixed_mesh(out["s"].cpu().numpy(), 32, 64))


# ---- batches -----------------------------------------------------------------------------------
MEMBERS = [(200.0, 16, 32, 101), (300.0, 24, 48, 102), (200.0, 16, 32, 103), (256.0, 32, 64, 104),
           (300.0, 24, 48, 105)]


def make_batch(nstreams):
    from paper_1507_05329_gb300 import Batch, Params
    params = [Params(box=b, np_side=n, nmesh=m) for b, n, m, _ in MEMBERS]
    wns = [dev(cola_inputs.white_noise(n, seed=sd)) for _, n, _, sd in MEMBERS]
    return Batch(params, wns, nbins=32, nstreams=nstreams), params, wns


def single_runs(params, wns):
    from paper_1507_05329_gb300 import Context
    outs = []
    for p, w in zip(params, wns):
        ctx = Context(p)
        o = ctx.run(w, nbins=32)
        ctx.sync()
        outs.append({k: v.clone() for k, v in o.items()})
        ctx.close()
    return outs


@pytest.mark.parametrize("nstreams", [1, 3])
def test_batch_equals_single_runs_eager_and_graph(nstreams):
    batch, params, wns = make_batch(nstreams)
    ref = single_runs(params, wns)
    lanes = {batch.info(i)["lane"] for i in range(len(MEMBERS))}
    assert lanes == set(range(min(nstreams, len(MEMBERS))))
    batch.run(use_graph=False)
    batch.sync()
    for o, r in zip(batch.outputs, ref):
        for k in ("s", "v", "psi1", "psi2", "pk"):
            assert torch.equal(o[k], r[k]), k
    for o in batch.outputs:
        for k in ("s", "v", "pk"):
            o[k].zero_()
    batch.run(use_graph=True)    # warm-up run, capture, launch
    batch.sync()
    assert batch.info(0)["graph_nodes"] > 10 * len(MEMBERS)
    for o, r in zip(batch.outputs, ref):
        for k in ("s", "v", "psi1", "psi2", "pk"):
            assert torch.equal(o[k], r[k]), k
    for o in batch.outputs:
        o["s"].fill_(float("nan"))
    batch.run(use_graph=True)    # replay only
    batch.sync()
    for o, r in zip(batch.outputs, ref):
        assert torch.equal(o["s"], r["s"])
    batch.close()


def test_batch_member_matches_the_oracle():
    """The 32^3 / 64^3 member (seed 104) against the FP64 oracle run: final positions within 1e-3
    mesh cells RMS, the whole-run bar of the single-realisation parity tests."""
    batch, params, wns = make_batch(2)
    batch.run(use_graph=True)
    batch.sync()
    i = 3
    p = params[i]
    ref = cola.run(cola_inputs.white_noise(p.np_side, seed=MEMBERS[i][3]).astype(np.float64),
                   oracle.Params(box=p.box, np_side=p.np_side, nmesh=p.nmesh), nbins=32)
    got = batch.outputs[i]["s"].cpu().numpy().astype(np.float64)
    rms = np.sqrt(np.mean((got - ref["s"]) ** 2))
    assert rms < 1e-3
    batch.close()


def test_batch_tune_then_graph_still_matches():
    """After per-shape autotuning the graph is captured again; positions agree with the untuned
    single runs to FP32 rounding-order differences (< 1e-4 cells RMS), P(k) to 1e-4."""
    batch, params, wns = make_batch(3)
    ref = single_runs(params, wns)
    batch.run(use_graph=True)
    batch.sync()
    batch.tune(reps=2)
    shapes = {}
    for i, p in enumerate(params):
        shapes.setdefault((p.np_side, p.nmesh), set()).add(batch.info(i)["schedule"])
    assert all(len(v) == 1 for v in shapes.values())
    assert batch.info(0)["graph_nodes"] == 0   # dropped: the next graph run captures again
    batch.run(use_graph=True)
    batch.sync()
    for o, r in zip(batch.outputs, ref):
        d = (o["s"] - r["s"]).double()
        assert float(d.pow(2).mean().sqrt()) < 1e-4
        m = r["pk"][2] > 0
        rel = ((o["pk"][1][m] - r["pk"][1][m]) / r["pk"][1][m]).abs().max()
        assert float(rel) < 1e-4
    batch.close()


def test_batch_rejects_bad_arguments():
    from paper_1507_05329_gb300 import Batch, ColaError, Params
    p = Params(box=100.0, np_side=16, nmesh=32)
    w = dev(cola_inputs.white_noise(16, seed=1))
    with pytest.raises(ColaError):
        Batch([p], [w], nbins=0)
    with pytest.raises(ColaError):
        Batch([p], [w], nstreams=0)
