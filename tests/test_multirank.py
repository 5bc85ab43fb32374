"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): max-over-ranks timing,
whole-job sums, disjoint sharding of independent units, and rank-0-only reporting."""
import io
import os
import socket
import contextlib

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        mx = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        sm = bench.sum_over_ranks(rank + 1, dist, "cpu")
        mine = bench.shard(range(11), rank, world)
        q.put((rank, mx, sm, mine))
    finally:
        dist.destroy_process_group()


def test_two_rank_reductions_and_sharding():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [20.0, 20.0]     # the job time is the slowest rank's
    assert [o[2] for o in out] == [3.0, 3.0]       # whole-job totals
    shards = [set(o[3]) for o in out]
    assert shards[0].isdisjoint(shards[1]) and shards[0] | shards[1] == set(range(11))


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class A:
        gpus, steps, warmup = 2, 1, 1
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A(), bench.WORKLOADS["d3q19_256_f32"], rank=1)
    assert buf.getvalue() == ""
