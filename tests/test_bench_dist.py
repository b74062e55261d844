"""The benchmark's multi-rank logic on CPU: two gloo ranks (no GPU).

Under torchrun every rank checks its own units (replicas of the instance, or
its shard of the batch's kernels) with no exchange on the data path; the
only collectives are the reductions of times (max over ranks) and counts
(sum over ranks) that make the reported whole-job numbers."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_max, e_max = bench.combine([10.0 + rank, 3.0 - rank], dist, "max")
        acc, n = bench.combine([100 * (rank + 1), 7], dist, "sum")
        q.put((rank, t_max, e_max, acc, n, list(bench.shard(10, rank, world))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, e_max, acc, n, sh in res:
        assert (t_max, e_max) == (11.0, 3.0)      # the slowest rank's times
        assert (acc, n) == (300.0, 14.0)          # whole-job totals
    shards = [r[5] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(10)) and not set(shards[0]) & set(shards[1])


def test_single_process_is_identity():
    import bench
    assert bench.combine([1.5, 2.0], None, "max") == [1.5, 2.0]
    assert list(bench.shard(5, 0, 1)) == [0, 1, 2, 3, 4]


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched as two ranks: rank 0 times the
    oracle and prints the one JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    port = _free_port()
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [x for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
