"""The benchmark's multi-rank logic on CPU with gloo (world size 2): timings are
maximised over ranks and the whole-job rate counts every rank's units; under
torchrun the reference arm prints one line from rank 0 and every rank exits 0."""

import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [10.0 + 5.0 * rank, 3.0 - rank]        # rank 1 is slower on the first timing
        got = bench.over_ranks(ms, dist, device="cpu")
        out[rank] = (got, bench.whole_job_rate(20, world, got[0]))
    finally:
        dist.destroy_process_group()


def test_over_ranks_takes_the_slowest_rank_and_counts_every_rank():
    import random

    port = 29500 + random.randint(0, 2000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        got, rate = res[rank]
        assert got == [15.0, 3.0]
        assert rate == pytest.approx(2 * 20 / 0.015)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.over_ranks([1.5, 2.5], None) == [1.5, 2.5]
    assert bench.whole_job_rate(10, 1, 1000.0) == pytest.approx(10.0)


def test_reference_arm_under_torchrun_prints_once():
    import random

    port = 29500 + random.randint(2001, 4000)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "tiny"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
