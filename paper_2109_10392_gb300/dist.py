"""Multi-GPU pieces of the batch optimizer (one process per GPU).

Trajectories of one scene are independent given the scene (Remark 1), and so
are scenes; the path therefore shards without any exchange on the data path.
What remains global is the choice of the best trajectory (Sec. III-F): when a
scene's goals are split across ranks, each rank scores its share (mmpc_score
gives its local argmin) and one MINLOC all-reduce of (meta cost, global goal
index) picks the scene's argmin -- 8 bytes per rank.  The key packs the
cost's IEEE bits (costs are >= 0, so the bits order like the values) above
the global index, as the scoring kernels do, so ties go to the lowest global
index and a rank with no finite cost contributes +inf.

`aggregate` is the whole-job timing rule of the benchmark: units summed over
ranks, time = the slowest rank.
"""
from __future__ import annotations

import math
import struct

NO_KEY = (1 << 63) - 1  # int64 max: +inf cost (all-rejected) on this rank


def shard(B: int, world: int, rank: int) -> tuple[int, int]:
    """[begin, end) of rank's share of B goals (contiguous, sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world or B < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(B, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def pack_key(cost: float, global_index: int) -> int:
    """int64 key ordering by (cost, index); NaN, +inf or a negative index -> NO_KEY."""
    if global_index < 0 or not math.isfinite(cost) or math.isnan(cost):
        return NO_KEY
    bits = struct.unpack("<I", struct.pack("<f", max(float(cost), 0.0)))[0]
    return (bits << 31) | (global_index & 0x7FFFFFFF)


def unpack_key(key: int) -> tuple[float, int]:
    if key == NO_KEY:
        return math.inf, -1
    bits, idx = key >> 31, key & 0x7FFFFFFF
    return struct.unpack("<f", struct.pack("<I", bits))[0], idx


def global_argmin(local_cost: float, local_index: int, offset: int, group=None, device=None) -> tuple[float, int]:
    """Scene argmin over all ranks: each rank passes its local argmin
    (local_index = -1 when every local trajectory was rejected) and the
    offset of its share; returns (cost, global index), (+inf, -1) if none."""
    import torch
    import torch.distributed as dist
    gi = offset + local_index if local_index >= 0 else -1
    t = torch.tensor([pack_key(local_cost, gi)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return unpack_key(int(t.item()))


def aggregate(units: float, ms: float, group=None, device=None) -> tuple[float, float]:
    """(units summed over ranks, max over ranks of ms)."""
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(t.item())
