"""Host-side logic of bench.py's multi-GPU mode (replicas only: one independent realisation per rank,
no collective on the data path), run as two gloo ranks on the CPU: distinct seeds per rank, the
slowest rank's time is the job's time, and the whole-job rate sums the ranks' particle-steps."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank                        # rank 1 is the slower one
    slow = bench.slowest_rank_ms(ms, dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(3, rank))
    out[rank] = (slow, seeds, bench.whole_job_rate(world, 1000, 10, slow))
    dist.destroy_process_group()


def test_two_replicas_on_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slow, seeds, rate = res[rank]
        assert slow == 150.0
        assert len(set(seeds)) == world
        assert rate == pytest.approx(2 * 1000 * 10 / 0.150)


def test_bench_gpus_n_starts_n_ranks():
    """`python bench.py --gpus 2` started by hand (no WORLD_SIZE) re-runs itself as two ranks under
    torch.distributed.run; --launch-check makes every rank join a gloo group and report, no GPU work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--launch-check"],
                         capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [json.loads(ln) for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    line = lines[0]
    assert line["launch_check"] is True and line["n_gpus"] == 2
    assert sorted(r["rank"] for r in line["ranks"]) == [0, 1]
    assert len({r["pid"] for r in line["ranks"]}) == 2
