"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The single-molecule workload runs as independent replicas and the batched
workload shards its molecules over the ranks; both report the slowest rank's
time and the sum of the ranks' interactions.  No GPU is involved.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, costs, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, count = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 * (rank + 1), "cpu")
        mine = bench.shard_molecules(costs, world, rank)
        out.put((rank, ms, count, mine))
    finally:
        dist.destroy_process_group()


def test_reduce_and_shard_over_two_gloo_ranks():
    costs = [float(a) ** (4.0 / 3.0) for a in (50, 3000, 120, 900, 2500, 75, 400, 1800, 60, 1300)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, count, _ in res:
        assert ms == 20.0          # max over ranks
        assert count == 3000.0     # sum over ranks
    shards = [set(r[3]) for r in res]
    assert shards[0].isdisjoint(shards[1])
    assert shards[0] | shards[1] == set(range(len(costs)))
    loads = [sum(costs[m] for m in s) for s in shards]
    assert max(loads) / min(loads) < 1.3, loads


def test_single_process_passthrough_and_shards():
    assert bench.reduce_over_ranks(3.5, 7, "cpu") == (3.5, 7.0)
    costs = [5.0, 1.0, 4.0, 2.0, 3.0]
    assert bench.shard_molecules(costs, 1, 0) == [0, 1, 2, 3, 4]
    parts = [bench.shard_molecules(costs, 3, r) for r in range(3)]
    assert sorted(m for p in parts for m in p) == [0, 1, 2, 3, 4]
    # longest first: 5 -> r0, 4 -> r1, 3 -> r2, 2 -> r2 (load 3 < 4 < 5), 1 -> r1 (4 < 5)
    assert parts == [[0], [1, 2], [3, 4]]
