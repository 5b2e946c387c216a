"""The multi-rank path on CPU: two gloo ranks (one process each).

* goal sharding covers the batch exactly once;
* the scene argmin over ranks (MINLOC all-reduce of packed (cost, global
  index) keys) equals the argmin of the whole batch under the scoring rules:
  lowest cost, ties to the lowest global index, NaN and +inf rejected, -1 when
  every trajectory is rejected;
* the benchmark's whole-job aggregation: units summed, time = slowest rank.
"""
import math
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2109_10392_gb300 import dist as D


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _local_argmin(c):
    best, idx = math.inf, -1
    for i, v in enumerate(c):
        if math.isfinite(v) and v < best:
            best, idx = v, i
    return best, idx


def _rank_main(rank, world, port, cases, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    for costs in cases:
        b, e = D.shard(len(costs), world, rank)
        c, i = _local_argmin(costs[b:e])
        out.append(D.global_argmin(c, i, b))
    u, t = D.aggregate(100.0 * (rank + 1), 3.0 + rank)
    out.append((u, t))
    import bench
    agg = bench.combine_ranks(dict(units=10.0 + rank, ms=1.0 + 2 * rank, e2e_units=5.0, e2e_ms=7.0 - rank), world, dist)
    out.append(agg)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def _run(world, cases):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, cases, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_shard_covers_batch():
    for B in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            got = [D.shard(B, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == B
            for (b0, e0), (b1, e1) in zip(got, got[1:]):
                assert e0 == b1
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1


def test_key_order():
    assert D.pack_key(1.0, 5) < D.pack_key(1.0, 6) < D.pack_key(1.5, 0) < D.NO_KEY
    assert D.pack_key(float("nan"), 0) == D.NO_KEY and D.pack_key(math.inf, 0) == D.NO_KEY
    assert D.unpack_key(D.pack_key(2.5, 17)) == (2.5, 17)
    assert D.unpack_key(D.NO_KEY) == (math.inf, -1)


@pytest.mark.timeout(300)
def test_two_gloo_ranks():
    rng = np.random.default_rng(0)
    cases = [list(rng.uniform(0, 10, 11)),
             [3.0, 1.0, 2.0, 1.0, 5.0, 1.0],                       # ties across the shard boundary
             [math.inf, float("nan"), math.inf, 4.0, math.inf],     # rejected trajectories
             [math.inf, math.inf, float("nan")],                    # every trajectory rejected
             [7.0],                                                 # rank 1 holds nothing
             list(rng.uniform(0, 1, 1000).astype(np.float32).astype(float))]
    res = _run(2, cases)
    for r in (0, 1):
        out = res[r]
        for costs, got in zip(cases, out[:len(cases)]):
            want_c, want_i = _local_argmin(costs)
            assert got[1] == want_i, (costs, got)
            if want_i >= 0:
                assert got[0] == np.float32(want_c)
        assert out[len(cases)] == (300.0, 4.0)
        agg = out[len(cases) + 1]
        assert agg["units"] == 21.0 and agg["ms"] == 3.0 and agg["e2e_units"] == 10.0 and agg["e2e_ms"] == 7.0
