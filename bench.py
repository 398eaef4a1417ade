"""Benchmark of the COLA particle-mesh hot path on GB300.

One step = one whole realisation through the public API (cola_run): 2LPT initial conditions,
10 COLA PM steps (deposit, FFTs, Poisson + gradient, three inverse FFTs, gather + kick + drift)
and the P(k) of the final positions.  Default workload: 1024^3 particles, 1536^3 PM mesh,
L = 1200 Mpc/h (flat LCDM Om=0.27, h=0.7, ns=0.96, sigma8=0.8, BBKS), seeded synthetic white noise.
Metric: particle-steps/s = (ranks x particles x 10 PM steps) / wall time of one realisation.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

--impl reference times the FP64 CPU oracle (the only reference this method has) on the host cores,
one oracle PM step per step, on a bounded sample of the same resolution (see SAMPLE).
With N > 1 (torchrun) every rank runs an independent realisation (different seed, no collective on
the data path): weak scaling, replicas only.
"""

from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import cola_inputs  # noqa: E402

METRIC = "particle-steps/s per PM step (whole realisation: 2LPT IC + 10 COLA steps + P(k))"
UNIT = "particle-steps/s"
WORKLOADS = {
    "large": dict(box=1200.0, np_side=1024, nmesh=1536, seed=3),
    "medium": dict(box=600.0, np_side=256, nmesh=512, seed=2),
    "small": dict(box=256.0, np_side=32, nmesh=64, seed=1),
    # the large workload's cell size and r = 1.5 in a 300 Mpc/h box (about 2 GB): ncu captures
    "profile": dict(box=300.0, np_side=256, nmesh=384, seed=3),
}
# CPU oracle sample: same mesh cell (L/N = 0.78 Mpc/h), same r = N/Np = 1.5 as the large workload
SAMPLE = dict(box=150.0, np_side=128, nmesh=192, seed=3)
L2_BYTES = 129 * 2 ** 20


def describe(w):
    return (f"{w['np_side']}^3 particles, {w['nmesh']}^3 PM mesh, L={w['box']:g} Mpc/h, 10 COLA steps, "
            f"seed {w['seed']}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


# ---- replicas: one independent realisation per rank, no collective on the data path ---------------
def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's realisation: independent white noise per replica."""
    return base_seed + 1000 * rank


def slowest_rank_ms(ms: float, dist, device) -> float:
    """Max over ranks of a per-rank time (the only collective: one scalar after the timed region)."""
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, particles: int, nstep: int, ms: float) -> float:
    """Particle-steps per second of all replicas together, timed by the slowest rank."""
    return world * particles * nstep / (ms / 1e3)


# ---- algorithmic bytes per launch of each stage (mesh N, particles n) ---------------------------
def stage_bytes(n_mesh: int, n_part: int, binned: bool = True) -> dict:
    """Bytes each stage must move once.  The tile (binned) deposit sums the exact fixed-point mesh in
    shared memory and writes the float density contrast (4 B per cell), which the z pass reads; the
    direct deposit writes and the z pass reads the 8-byte fixed-point mesh."""
    nc = n_mesh // 2 + 1
    cplx = 8.0 * n_mesh * n_mesh * nc          # one complex half-spectrum field
    real = 4.0 * n_mesh ** 3                   # one real field
    mesh = (4.0 if binned else 8.0) * n_mesh ** 3
    return {
        "deposit": 12.0 * n_part + mesh,
        "fwd_z_r2c": mesh + cplx,
        "fwd_y": 2 * cplx,
        "green_x": cplx + 3 * cplx,
        "inv_y": 2 * cplx,
        "inv_z_c2r": cplx + real,
        "gather_kick_drift": 3 * real + 48.0 * n_part + 24.0 * n_part,
    }


# ---- nvidia-smi clock sampler --------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU oracle baseline (the FP64 oracle as it stands, on the host cores) ----------------------
# The oracle is plain single-threaded numpy; it uses the host's cores through independent replicas
# (one process per core, each its own realisation), the same parallelism as the GPU arm's replicas.
# Processes are started with `spawn` (never forked from a process that has touched the GPU).
CPU_CONFIGS = {
    "32^3/64^3": dict(box=256.0, np_side=32, nmesh=64, seed=1),      # the small parity workload
    "256^3/512^3": dict(box=600.0, np_side=256, nmesh=512, seed=2),  # the medium workload
}
ORACLE_BYTES_PER_MESH_CELL = 90.0   # peak host memory of one oracle step per mesh cell (11.3 GB at 512^3)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_available_bytes() -> float:
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return float(line.split()[1]) * 1024.0
    except OSError:
        pass
    return 16e9


def _oracle_worker(conn, w, seed):
    """One oracle replica: set up its realisation, then one timed COLA step per request."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle
    from oracle import cola, lpt, rng
    p = oracle.Params(box=w["box"], np_side=w["np_side"], nmesh=w["nmesh"])
    psi1, psi2 = lpt.displacements(rng.white_noise(seed, p.np_side), p)
    s, v = cola.initial_state(psi1, psi2, p)
    i = 0
    conn.send("ready")
    while conn.recv() == "step":
        t0 = time.perf_counter()
        s, v = cola.step(1 + i % p.nstep, s, v, psi1, psi2, p)
        conn.send(time.perf_counter() - t0)
        i += 1


class OracleReplicas:
    """`procs` oracle processes, each holding one realisation of workload w; step() advances them
    all by one COLA step concurrently and returns the wall time."""

    def __init__(self, w, procs: int):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for r in range(procs):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, w, w["seed"] + 1000 * r), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        for c in self.conns:
            c.recv()

    def step(self) -> float:
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("step")
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send("stop")
        for pr in self.procs:
            pr.join(timeout=30)


def oracle_procs_for(w, cores: int) -> int:
    """Replicas that fit: one per core, at most what half the available host memory holds."""
    per = ORACLE_BYTES_PER_MESH_CELL * w["nmesh"] ** 3
    return max(1, min(cores, int(0.5 * host_available_bytes() // per)))


def _oracle_parts_job(w):
    """Seconds of the particle work (deposit, interpolation) and of the mesh work (FFTs, Green
    function) of one oracle PM force at workload w, from the oracle's own functions."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle
    from oracle import cic, cola, lpt, pm, rng
    p = oracle.Params(box=w["box"], np_side=w["np_side"], nmesh=w["nmesh"])
    psi1, psi2 = lpt.displacements(rng.white_noise(w["seed"], p.np_side), p)
    s, _ = cola.initial_state(psi1, psi2, p)
    t0 = time.perf_counter()
    delta = pm.density_fixed(s, p.np_side, p.nmesh)
    t1 = time.perf_counter()
    f = pm.force_mesh(delta, 1.0)
    t2 = time.perf_counter()
    cell, w1 = cic.interp_weights_fixed(s, p.np_side, p.nmesh)
    cic.cic_interp(f, cell, w1)
    t3 = time.perf_counter()
    return {"particle_s": (t1 - t0) + (t3 - t2), "mesh_s": t2 - t1}


def _oracle_realisation_job(w):
    """Seconds of one oracle realisation's parts at workload w: 2LPT, one COLA step, one P(k)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle
    from oracle import cola, lpt, pm, power, rng
    p = oracle.Params(box=w["box"], np_side=w["np_side"], nmesh=w["nmesh"])
    t0 = time.perf_counter()
    psi1, psi2 = lpt.displacements(rng.white_noise(w["seed"], p.np_side), p)
    t1 = time.perf_counter()
    s, v = cola.initial_state(psi1, psi2, p)
    s, v = cola.step(1, s, v, psi1, psi2, p)
    t2 = time.perf_counter()
    power.power_spectrum(pm.density_fixed(s, p.np_side, p.nmesh), p.box, 64)
    t3 = time.perf_counter()
    return {"ic_s": t1 - t0, "step_s": t2 - t1, "pk_s": t3 - t2}


def _oracle_adjoint_job(args):
    """Seconds of the oracle's forward (2LPT + 10 steps, continuous CIC) or forward + adjoint."""
    w, ngrid, which = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    import oracle
    from oracle import adjoint, rng
    p = oracle.Params(box=w["box"], np_side=w["np_side"], nmesh=w["nmesh"])
    wn = rng.white_noise(w["seed"], p.np_side)
    t0 = time.perf_counter()
    if which == "forward":
        adjoint.forward(wn, p)
    else:
        adjoint.gradient(wn, p, ngrid, np.zeros((ngrid,) * 3))
    return time.perf_counter() - t0


def cpu_baseline_entry():
    """The FP64 oracle on the host cores: particle-steps/s per PM step at 32^3/64^3 and 256^3/512^3
    (one replica per core, within host memory), the 1024^3/1536^3 rate extrapolated from the
    256^3/512^3 step, and CPU estimates of the batched mocks/hour and the adjoint/forward cost.  The
    side measurements (six processes) run beside the 256^3/512^3 replicas, on cores of their own."""
    import multiprocessing as mp
    cores = host_cores()
    out = {"kind": "oracle", "unit": UNIT, "cores": cores, "nproc": cores}
    rates = {}
    small = CPU_CONFIGS["32^3/64^3"]
    procs = oracle_procs_for(small, cores)
    reps = OracleReplicas(small, procs)
    t = min(reps.step() for _ in range(3))
    reps.close()
    rates["32^3/64^3"] = {"value": procs * small["np_side"] ** 3 / t, "processes": procs, "step_wall_s": t}
    med = CPU_CONFIGS["256^3/512^3"]
    side = 6
    mem_slots = int(0.5 * host_available_bytes() // (ORACLE_BYTES_PER_MESH_CELL * med["nmesh"] ** 3))
    procs = max(1, min(cores - side, mem_slots - 1))
    with mp.get_context("spawn").Pool(side) as pool:
        parts_r = pool.apply_async(_oracle_parts_job, (med,))
        shapes = [dict(box=300.0, np_side=96, nmesh=192, seed=100), dict(box=400.0, np_side=128, nmesh=256, seed=124),
                  dict(box=500.0, np_side=160, nmesh=320, seed=148)]
        real_r = [pool.apply_async(_oracle_realisation_job, (w,)) for w in shapes]
        adj_w = dict(box=200.0, np_side=64, nmesh=128, seed=4)   # the differentiable workload's cell, 1/8 volume
        fwd_r = pool.apply_async(_oracle_adjoint_job, ((adj_w, 32, "forward"),))
        grad_r = pool.apply_async(_oracle_adjoint_job, ((adj_w, 32, "gradient"),))
        reps = OracleReplicas(med, procs)
        t = reps.step()
        reps.close()
        rates["256^3/512^3"] = {"value": procs * med["np_side"] ** 3 / t, "processes": procs, "step_wall_s": t}
        parts = parts_r.get()
        reals = [r.get() for r in real_r]
        fwd_s, grad_s = fwd_r.get(), grad_r.get()
    # 1024^3 / 1536^3: the particle work scales with n, the mesh work with N^3 log N^3
    n1, N1, n2, N2 = med["np_side"] ** 3, med["nmesh"], 1024 ** 3, 1536
    step1 = rates["256^3/512^3"]["step_wall_s"]
    other = max(step1 - parts["particle_s"] - parts["mesh_s"], 0.0)
    mesh_scale = (N2 ** 3 * math.log2(N2 ** 3)) / (N1 ** 3 * math.log2(N1 ** 3))
    t_large = (parts["particle_s"] + other) * n2 / n1 + parts["mesh_s"] * mesh_scale
    # CPU mocks/hour: realisation = 2LPT + 10 steps + P(k) per shape, the 64-member mix over all cores
    per_shape = [r["ic_s"] + 10.0 * r["step_s"] + r["pk_s"] for r in reals]
    batch_cpu_s = 24 * per_shape[0] + 24 * per_shape[1] + 16 * per_shape[2]
    out.update({
        "value": rates["256^3/512^3"]["value"],
        "sample": ("FP64 numpy oracle, one COLA step per replica process, one replica per core within host memory: "
                   "value = 256^3 particles / 512^3 mesh (600 Mpc/h), processes in by_config"),
        "by_config": rates,
        "large_extrapolated": {"value": cores * n2 / t_large, "seconds_per_step_one_core": t_large,
                               "note": "extrapolated, not run: 1024^3/1536^3 needs ~300 GB of FP64 meshes; particle "
                                       "work scaled by n, mesh work by N^3 log N^3 from the 256^3/512^3 step, all cores "
                                       "as independent replicas"},
        "batched_mocks_per_hour_estimated": 64 * 3600.0 * cores / batch_cpu_s,
        "batched_note": "estimated from one timed 2LPT, COLA step and P(k) per shape (96^3/192^3, 128^3/256^3, "
                        "160^3/320^3); realisation = 2LPT + 10 steps + P(k); 64-member mix over all cores",
        "adjoint_over_forward": (grad_s - fwd_s) / fwd_s,
        "adjoint_note": "oracle forward (2LPT + 10 steps) vs forward + hand-written adjoint, 64^3/128^3 in 200 Mpc/h "
                        "(the differentiable workload's cell), loss on a 32^3 grid",
    })
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    cores = host_cores()
    procs = oracle_procs_for(SAMPLE, cores)
    reps = OracleReplicas(SAMPLE, procs)
    for _ in range(args.warmup):
        reps.step()
    timed = [reps.step() for _ in range(args.steps)]
    reps.close()
    t = sum(timed) / len(timed)
    value = procs * SAMPLE["np_side"] ** 3 / t
    sample = (f"{procs} FP64 oracle replicas (one process per core), one COLA step each per step, on "
              f"{describe(SAMPLE)}: the large workload's cell size and particle spacing in a smaller box")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(w), "timed_sample": describe(SAMPLE), "nproc": cores},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- our arm -------------------------------------------------------------------------------------
def source_digest() -> str:
    h = hashlib.sha256()
    for f in ("fft.cu", "fft_core.cuh", "fft_fast.inc", "particles.cu", "binning.cu"):   # the PM-step kernels
        with open(os.path.join(ROOT, "paper_1507_05329_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(stage: str, workload: str):
    """DRAM bytes per launch of `stage` from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_digest") != source_digest():
        return None
    ent = rec.get("stages", {}).get(stage)
    if not ent:
        return None
    return ent.get("dram_bytes_per_launch_" + workload)


def measure_adjoint(args, torch, device):
    """Adjoint cost against the plain forward on the differentiable workload (400 Mpc/h, 128^3
    particles, 256^3 mesh, seed 4, loss on a 64^3 CIC grid against the seed-5 realisation).
    forward = cola_run without P(k); backward = loss-grid adjoint + cola_adjoint (10 force
    recomputations from the per-step checkpoints).  The working set (about 0.9 GB) exceeds L2."""
    from paper_1507_05329_gb300 import Context, Params
    wl = cola_inputs.WORKLOADS["adjoint"]
    cfg = cola_inputs.ADJOINT_LOSS
    from paper_1507_05329_gb300 import binding
    p = Params(box=wl["box"], np_side=wl["np_side"], nmesh=wl["nmesh"], nstep=10, seed=wl["seed"])
    stream = torch.cuda.current_stream()
    ctx = Context(p, stream)
    ng = cfg["ngrid"]
    wn = binding.white_noise(p)                                   # the library's seeded field
    tgt = ctx.grid_density(ctx.run(binding.white_noise(dataclasses.replace(p, seed=cfg["target_seed"])),
                                   with_pk=False)["s"], ng)
    out = {k: ctx.empty_particles() for k in ("s", "v", "psi1", "psi2")}

    def timed(fn, k):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    k = max(args.steps, 3)
    fwd_ms = timed(lambda: ctx.run(wn, with_pk=False, out=out), k)
    state = {}

    def fwd_ckpt():
        state["f"] = ctx.run_checkpointed(wn)
        state["d"] = ctx.grid_density(state["f"]["s"], ng)

    ck_ms = timed(fwd_ckpt, k)
    lam_d = (2.0 * (state["d"] - tgt)).contiguous()

    def backward():
        lam_s = ctx.grid_density_adjoint(state["f"]["s"], ng, lam_d)
        state["g"] = ctx.adjoint(wn, state["f"]["ckpt"], lam_s)

    bwd_ms = timed(backward, k)
    ctx.sync()
    ctx.close()
    return {"workload": f"{p.np_side}^3 particles, {p.nmesh}^3 PM mesh, L={p.box:g} Mpc/h, 10 COLA steps, "
                        f"loss on a {ng}^3 CIC grid, seeds {wl['seed']}/{cfg['target_seed']}",
            "forward_ms": fwd_ms, "forward_checkpointed_ms": ck_ms, "backward_ms": bwd_ms,
            "adjoint_over_forward": bwd_ms / fwd_ms,
            "forward_plus_backward_over_forward": (ck_ms + bwd_ms) / fwd_ms, "steps": k}


def measure_batched(args, torch, device):
    """Batched mocks: the 64 uneven realisations (24 x 96^3/192^3/300, 24 x 128^3/256^3/400,
    16 x 160^3/320^3/500 Mpc/h, seeds 100-163, 10 COLA steps and P(k) each).  Plain = one
    realisation after another through cola_run on one stream; batched = cola_batch over
    `--lanes` streams, autotuned per shape, replayed from one captured CUDA graph.  The working
    set (about 30 GB) exceeds L2."""
    from paper_1507_05329_gb300 import Batch, Context, Params
    members = cola_inputs.batched_workload()
    params = [Params(box=m["box"], np_side=m["np_side"], nmesh=m["nmesh"], nstep=10, seed=m["seed"]) for m in members]
    from paper_1507_05329_gb300 import binding
    fields = [binding.white_noise(p) for p in params]   # the plain loop's inputs: each member's seeded field
    stream = torch.cuda.current_stream()
    k = max(args.steps, 2)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # plain: one context per shape, realisations in sequence
    ctxs = {}
    for p in params:
        if (p.np_side, p.nmesh, p.box) not in ctxs:
            ctxs[(p.np_side, p.nmesh, p.box)] = Context(p, stream)
    outs = {key: {n: c.empty_particles() for n in ("s", "v", "psi1", "psi2")} for key, c in ctxs.items()}
    for key, o in outs.items():
        o["pk"] = torch.empty((3, 64), dtype=torch.float64, device=device)

    def plain():
        for p, w in zip(params, fields):
            key = (p.np_side, p.nmesh, p.box)
            ctxs[key].run(w, 64, out=outs[key])

    plain_ms = timed(plain, k)
    for c in ctxs.values():
        c.sync()
        c.close()
    del ctxs, outs
    torch.cuda.empty_cache()

    del fields
    # batched: every member draws the field of its own seed inside its cola_run (white noise None)
    batch = Batch(params, [None] * len(params), nbins=64, nstreams=args.lanes, stream=stream)
    batch.run(use_graph=False)
    batch.sync()
    batch.tune(reps=5)          # force evaluations of 1-3 ms: more repetitions than the large workload's 2
    batch.run(use_graph=True)   # warm-up + capture + launch
    batch.sync()
    graph_ms = timed(lambda: batch.run(use_graph=True), k)
    eager_ms = timed(lambda: batch.run(use_graph=False), k)
    batch.sync()
    info = [batch.info(i) for i in range(len(params))]
    scheds = {}
    for p, inf in zip(params, info):
        scheds[f"{p.np_side}^3/{p.nmesh}^3"] = inf["schedule"]
    batch.close()
    n = len(params)
    return {"workload": "64 realisations: 24 x (96^3, 192^3, 300 Mpc/h), 24 x (128^3, 256^3, 400), "
                        "16 x (160^3, 320^3, 500), seeds 100-163, 10 COLA steps + P(k) each",
            "mocks_per_hour": n * 3.6e6 / graph_ms, "graph_ms_per_batch": graph_ms,
            "plain_mocks_per_hour": n * 3.6e6 / plain_ms, "plain_ms_per_batch": plain_ms,
            "eager_lanes_ms_per_batch": eager_ms, "speedup_vs_plain": plain_ms / graph_ms,
            "lanes": args.lanes, "graph_nodes": info[0]["graph_nodes"], "schedules": scheds, "steps": k}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1507_05329_gb300 import Context, Params, build, binding

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    w = WORKLOADS[args.workload]
    seed = replica_seed(w["seed"], rank)
    p = Params(box=w["box"], np_side=w["np_side"], nmesh=w["nmesh"], nstep=10, seed=seed)
    n = p.n
    stream = torch.cuda.current_stream()
    ctx = Context(p, stream)
    wn = None          # each realisation draws the field of its seed (Philox-4x32-10) inside cola_run
    out = {k: ctx.empty_particles() for k in ("s", "v", "psi1", "psi2")}
    out["pk"] = torch.empty((3, args.nbins), dtype=torch.float64, device=f"cuda:{local}")

    def barrier():
        if ws > 1:
            dist.barrier()

    tuned = None
    if args.schedule is not None:
        ctx.schedule = args.schedule   # fixed for every realisation, warm-up included
        tuned = {"schedule": args.schedule, "force_eval_ms": None, "fixed": True}
    for _ in range(args.warmup):
        ctx.run(wn, args.nbins, out=out)
    ctx.sync()
    if args.autotune and args.schedule is None:
        # schedule chosen on the evolved (a = 1) positions of the warm-up realisation; outside the timed region
        best, times = ctx.autotune(out["s"], reps=2)
        tuned = {"schedule": best, "force_eval_ms": {str(k): round(v, 3) for k, v in times.items()}}
        ctx.run(wn, args.nbins, out=out)
        ctx.sync()

    ctx_schedule = ctx.schedule
    # kernels per realisation, counted from a captured (unexecuted) graph of the same cola_run call
    kernels_per_run = ctx.run_kernel_count(wn, args.nbins, out=out)
    ctx.sync()
    sampler = ClockSampler(local)
    ctx.profile(True)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.run(wn, args.nbins, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ctx.sync()
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        ms = slowest_rank_ms(ms, dist, f"cuda:{local}")
    value = whole_job_rate(ws, n, p.nstep, ms)
    me = {"rank": rank, "local_rank": local, "device": torch.cuda.get_device_name(local),
          "pci_bus_id": torch.cuda.get_device_properties(local).pci_bus_id if hasattr(
              torch.cuda.get_device_properties(local), "pci_bus_id") else None}
    rank_devices = [me]
    if ws > 1:
        rank_devices = [None] * ws
        dist.all_gather_object(rank_devices, me)

    # roofline of the dominant PM-step kernel
    sb = stage_bytes(p.nmesh, n, binned=bool(ctx_schedule & binding.SCHED_BINNED_DEPOSIT))
    stages = {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items()}
    pm_stages = [k for k in sb if prof[k][1] > 0]
    dom = max(pm_stages, key=lambda k: prof[k][0])
    avg_ms = prof[dom][0] / prof[dom][1]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = sb[dom] / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "traffic": recorded_traffic(dom, args.workload),
                "traffic_source": "ncu dram__bytes_read+write per launch from profiles/traffic.json"
                                  + (", scaled 64x from the 256^3/384^3 capture" if args.workload == "large" else ""),
                "algorithmic_bytes_per_launch": sb[dom], "avg_launch_ms": avg_ms}
    per_stage = {}
    for k in sb:
        if prof[k][1]:
            a = prof[k][0] / prof[k][1]
            per_stage[k] = {"avg_ms": round(a, 4), "launches": prof[k][1],
                            "GBps": round(sb[k] / (a / 1e3) / 1e9, 1), "frac": round(sb[k] / (a / 1e3) / 1e9 / peak, 3)}
    launches = kernels_per_run * args.steps
    if prof.get("bin", (0, 0))[1]:
        per_stage["bin"] = {"avg_ms": round(prof["bin"][0] / prof["bin"][1], 4), "launches": prof["bin"][1],
                            "note": "particle binning by mesh tiles (implementation overhead, not algorithmic bytes)"}
    pm_ms = sum(prof[k][0] for k in sb) / args.steps
    # every stage's device time per realisation (2LPT, PM steps, P(k)), CUDA events inside the timed region
    per_realisation = {k: round(v[0] / args.steps, 3) for k, v in prof.items() if v[1]}

    # end to end through the public API with host buffers (pinned), copies inside the timed region.
    # Realisation k's white noise goes in and its s, v, P(k) come out on a copy stream, overlapping the
    # neighbouring realisations' compute (double-buffered device inputs and outputs); the clock stops
    # when the last result has reached the host.
    e2e = None
    if args.e2e_steps > 0:
        # the user-supplied-field path of the public API: the seed's field travels from host memory
        wn_host = torch.empty(n, dtype=torch.float32, pin_memory=True)
        wn_host.copy_(binding.white_noise(p).cpu())
        s_host = torch.empty((3, n), dtype=torch.float32, pin_memory=True)
        v_host = torch.empty((3, n), dtype=torch.float32, pin_memory=True)
        pk_host = torch.empty((3, args.nbins), dtype=torch.float64, pin_memory=True)
        wn_dev = [torch.empty(n, dtype=torch.float32, device=f"cuda:{local}") for _ in range(2)]
        outs = [out, {"s": ctx.empty_particles(), "v": ctx.empty_particles(), "psi1": out["psi1"],
                      "psi2": out["psi2"], "pk": torch.empty_like(out["pk"])}]
        copy = torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_run = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(copy):
            wn_dev[0].copy_(wn_host, non_blocking=True)
            ev_in[0].record(copy)
        for k in range(args.e2e_steps):
            b = k % 2
            stream.wait_event(ev_in[b])
            if k >= 2:
                stream.wait_event(ev_out[b])          # realisation k-2's results have left buffer b
            ctx.run(wn_dev[b], args.nbins, out=outs[b])
            ev_run[b].record(stream)
            with torch.cuda.stream(copy):
                if k + 1 < args.e2e_steps:            # next input, while realisation k computes
                    if k >= 1:
                        copy.wait_event(ev_run[b ^ 1])    # realisation k-1 has finished with that buffer
                    wn_dev[b ^ 1].copy_(wn_host, non_blocking=True)
                    ev_in[b ^ 1].record(copy)
                copy.wait_event(ev_run[b])
                s_host.copy_(outs[b]["s"], non_blocking=True)
                v_host.copy_(outs[b]["v"], non_blocking=True)
                pk_host.copy_(outs[b]["pk"], non_blocking=True)
                ev_out[b].record(copy)
        copy.synchronize()
        torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / args.e2e_steps
        if ws > 1:
            t_e2e = slowest_rank_ms(t_e2e * 1e3, dist, f"cuda:{local}") / 1e3
        e2e = {"value": whole_job_rate(ws, n, p.nstep, t_e2e * 1e3), "unit": UNIT, "h2d_bytes_per_step": 4 * n,
               "d2h_bytes_per_step": 24 * n + 24 * args.nbins, "steps": args.e2e_steps,
               "ms_per_step": t_e2e * 1e3,
               "note": "copies on a second stream overlap the neighbouring realisations' compute; the first "
                       "input and the last output copy of the stream are not overlapped"}
        del wn_host, s_host, v_host, pk_host, wn_dev, outs

    ctx.sync()
    ctx.close()
    del out
    torch.cuda.empty_cache()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry()
    adj = batched = None
    if rank == 0 and not args.no_adjoint:
        adj = measure_adjoint(args, torch, f"cuda:{local}")
    if rank == 0 and not args.no_batched:
        batched = measure_batched(args, torch, f"cuda:{local}")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 (int64 fixed-point deposit)", "data": "synthetic",
                "config": {"workload": describe(w), "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                           "l2": "inputs larger than L2 (no flush needed)",
                           "pm_step_ms": pm_ms / 10.0, "nbins": args.nbins, "autotune": tuned,
                           "rank_devices": rank_devices},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "stages": per_stage, "ms_per_realisation_by_stage": per_realisation,
                "adjoint": adj, "batched": batched}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--nbins", type=int, default=64)
    ap.add_argument("--e2e-steps", type=int, default=8,
                    help="realisations in the end-to-end stream (the first input and the last output copies are "
                         "exposed once per stream)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward cost measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-mocks measurement")
    ap.add_argument("--lanes", type=int, default=8, help="streams of the batched-mocks run")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the size-based default schedule instead of timing the candidates first")
    ap.add_argument("--schedule", type=int, default=None,
                    help="run every realisation (warm-up included) under this cola_set_schedule value, untuned")
    ap.add_argument("--launch-check", action="store_true",
                    help="start the ranks (gloo, no GPU work) and print which ranks came up; no measurement")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return launch_ranks(args.gpus)
    if args.launch_check:
        return launch_check(args)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


def launch_ranks(n: int) -> int:
    """`bench.py --gpus N` started by hand: re-run this command as N local ranks (one per GPU) under
    torch.distributed.run on 127.0.0.1; rank 0 prints the line."""
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def launch_check(args) -> int:
    """Every rank joins a gloo group and reports (rank, local rank, world); rank 0 prints them."""
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("gloo")
        got = [None] * ws
        dist.all_gather_object(got, {"rank": rank, "local_rank": local, "pid": os.getpid()})
        dist.destroy_process_group()
    else:
        got = [{"rank": rank, "local_rank": local, "pid": os.getpid()}]
    if rank == 0:
        print(json.dumps({"launch_check": True, "n_gpus": ws, "ranks": got}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
