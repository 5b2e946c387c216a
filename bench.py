#!/usr/bin/env python3
"""Benchmark of the batch non-holonomic AM trajectory optimizer (arXiv
2109.10392, Algorithm 1 + meta-cost argmin) on GB300.

Default workload (--workload warm), the metric "trajectories/s to residual
<= 1e-2 m, warm-started vs plain GPU": 4096 fresh synthetic highway scenes x
256 goals (8 lateral offsets x 32 speeds ~ U(5, 30) m/s), 50 constant-velocity
obstacles, N = 100 samples, 12 Bernstein coefficients per axis, at most 100
AM iterations with early exit once a trajectory's residual is <= 1e-2 m
(checked every 10 iterations), FP32.  A network trained in the run on scenes
solved by the method itself gives the warm starts.  A step is one CUDA graph
replay of the target form over all scenes: features, network, decode, one
persistent solve launch, cold fallback of every miss, scoring, per-scene
argmin, with the opt-in stall stop.  `value` is the number of trajectories
that reach the residual target per second; `detail` holds the same figure for
the plain method (one mmpc_solve + mmpc_score per scene), the batched cold
start and every warm-start variant, with and without the stall stop, and the
plain 1024-goal scene's throughput.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                    [--workload warm|scene|batch|precision|sweep]

One JSON line on stdout (rank 0).  Each rank solves its own scenes: weak
scaling, no collective on the data path.  --impl reference times the FP64
CPU oracle (the plain cold-started method) on the host cores instead, on a
bounded sample of the same evaluation scenes per step, same stopping rule.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trajectories/s to residual<=1e-2 m, warm-started vs plain GPU; % of roofline"
STALL = (1.0, 0.5)  # opt-in stall stop: residual > 1 m and not halved over the last two checks
UNIT = "trajectories/s"
TOL = 1e-2
CHECK_EVERY = 10
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SFU_PER_SM = 16
SM_MAX_MHZ = 2070.0
FLUSH_BYTES = 256 << 20  # > 129 MB L2


def workload(seed: int, kind: str = "scene"):
    """scene: the 1024-goal, 50-obstacle scene (N = 100, n = 12); precision:
    16384 goals, 30 obstacles, N = 200, n = 16 (the same distribution)."""
    from paper_2109_10392_gb300 import scenes
    sc = scenes.scene_large(seed) if kind == "scene" else scenes.scene_custom(31 + seed, 16384, 30, N=200, n=16)
    params = dict(sc.params)
    params.update(tol=TOL, check_every=CHECK_EVERY)
    return sc, params


def workload_name(params, B, m):
    return f"highway_B{B}_m{m}_N{params['N']}_n{params['n']}_K{params['iters']}_tol{TOL:g}"


UNIT_CONV = "trajectories/s reaching residual <= 1e-2 m"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def _sha256_files(paths):
    import hashlib
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of `kernel` on `workload`, from
    the ncu figures recorded in profiles/dram_traffic.json, or None when no
    figure was taken with the kernel source as it is now (the entry stores
    the SHA-256 of the source files it was measured with)."""
    try:
        with open(TRAFFIC_FILE) as f:
            entries = json.load(f)["entries"]
    except (OSError, ValueError, KeyError):
        return None
    for e in entries:
        if e.get("kernel") == kernel and e.get("workload") == workload:
            try:
                src = e["source"] if isinstance(e["source"], list) else [e["source"]]
                if _sha256_files([os.path.join(ROOT, x) for x in src]) == e["sha256"]:
                    return e["bytes_per_launch"]
            except (OSError, KeyError):
                return None
    return None


OPS_PER_ELEMENT = 10  # FP32 lane ops per evaluated obstacle-sample pair


def alu_ops(N, n, passes, elements):
    """FP32 lane operations of a solve, per trajectory-iteration (every AM
    pass: the initial one and one per iteration run): 14 N n basis products
    (2 N n for xdot, ydot; N n for P^T theta; N n for psi; 4 N n for x, y,
    xddot, yddot; 6 N n for F^T g) + 7 n^2 for the QP and multiplier products
    + 60 N element-wise (velocity, heading trigonometry, acceleration
    projection, residuals), plus 10 per obstacle-sample pair of Eq.
    split_alpha_o (predicted offset 4, normalised squared distance 2,
    max(1/r - 1, 0) 2, accumulation 2).  `elements` = passes N m gives the
    algorithm's dense count (culled pairs are exact zeros); the evaluated
    pair count gives the work the kernel executed."""
    return elements * OPS_PER_ELEMENT + passes * (14 * N * n + 7 * n * n + 60 * N)


def tensor_peak_tflops(kind: str):
    """Dense tensor peak for `kind` from MEASURED_PEAKS.json's BF16 burst
    figure times the nominal ratio (TF32 1.1 / BF16 2.25 PFLOP/s); the
    recipe's fallback 1.9 PFLOP/s BF16 when the file is absent."""
    bf16 = 1900.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        for k in ("bf16_tflops", "bf16_dense_tflops"):
            if k in d:
                bf16 = float(d[k])
                break
    except (OSError, ValueError):
        pass
    return bf16 * (1.1 / 2.25 if kind == "tf32" else 1.0)


def rank_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def combine_ranks(local: dict, world: int, dist=None) -> dict:
    """Whole-job aggregate: units summed over ranks, time = max over ranks."""
    if world == 1 or dist is None:
        return dict(units=local["units"], ms=local["ms"], e2e_units=local["e2e_units"], e2e_ms=local["e2e_ms"])
    import torch
    t = torch.tensor([local["units"], local["e2e_units"]], dtype=torch.float64)
    mx = torch.tensor([local["ms"], local["e2e_ms"]], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t, mx = t.cuda(), mx.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    t, mx = t.cpu(), mx.cpu()
    return dict(units=float(t[0]), ms=float(mx[0]), e2e_units=float(t[1]), e2e_ms=float(mx[1]))


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except OSError:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def run_mine(args):
    import torch

    from paper_2109_10392_gb300 import mmpc

    rank, world, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    sc, params = workload(seed=rank, kind=args.workload)
    params["cull"] = 0 if args.no_cull else 1
    if args.stall:
        params.update(stall_tol=STALL[0], stall_ratio=STALL[1])
    params["variant"] = args.variant
    B, m, n = len(sc.goals), sc.obst.shape[0], params["n"]
    solver = mmpc.Solver(params, m)
    meta = mmpc.make_meta(**sc.meta)
    f32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev).contiguous()  # noqa: E731
    ego, obst, goals = f32(sc.ego), f32(sc.obst), f32(sc.goals)
    coef = torch.empty((B, 3 * n), dtype=torch.float32, device=dev)
    resid = torch.empty((B, 4), dtype=torch.float32, device=dev)
    iters = torch.empty((B,), dtype=torch.int32, device=dev)
    cost = torch.empty((B,), dtype=torch.float32, device=dev)
    argmin = torch.empty((1,), dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def solve():
        mmpc.mmpc_solve(solver.ctx, ego, obst, goals, coef, None, None, None, resid, iters, stream)

    def score():
        mmpc.mmpc_score(solver.ctx, meta, coef, cost, argmin, stream)

    for _ in range(args.warmup):
        flush.zero_()
        solve()
        score()
    torch.cuda.synchronize(dev)
    # the result of a step is deterministic: count converged trajectories once
    conv = (resid[:, :3].max(dim=1).values <= TOL)
    units_per_step = int(conv.sum().item())
    iters_sum = int(iters.to(torch.int64).sum().item())

    K = args.steps
    mmpc.mmpc_take_work_count(solver.ctx)  # reset the evaluated-pair counter
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(K):
        flush.zero_()  # L2 flush between timed steps (outside the event brackets)
        ev[i][0].record(stream)
        solve()
        ev[i][1].record(stream)
        score()
        ev[i][2].record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    elements = mmpc.mmpc_take_work_count(solver.ctx) / K  # per launch
    solve_ms = [e[0].elapsed_time(e[1]) for e in ev]
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    ms = sum(step_ms) / K
    solve_avg = sum(solve_ms) / K

    # end to end through the public API with host buffers: one mmpc_step_host
    # call per step copies the pinned inputs in, solves, scores, copies the
    # coefficients, residuals, costs and argmin back and waits for the stream
    Ke = min(K, args.e2e_steps)
    # one pinned block per direction, in the device order (ego, obstacles, goals /
    # coef, resid, cost): mmpc_step_host then makes one copy each way
    parts = [np.asarray(a, dtype=np.float32).reshape(-1) for a in (sc.ego, sc.obst.reshape(-1, 4), sc.goals)]
    blk_in = torch.from_numpy(np.concatenate(parts)).pin_memory()
    h_in = [blk_in[:4], blk_in[4:4 + 4 * m].view(m, 4), blk_in[4 + 4 * m:].view(-1, 3)]
    nc, nr = coef.numel(), resid.numel()
    blk_out = torch.empty(nc + nr + cost.numel(), dtype=torch.float32).pin_memory()
    h_out = [blk_out[:nc].view(coef.shape), blk_out[nc:nc + nr].view(resid.shape), blk_out[nc + nr:].view(cost.shape),
             torch.empty(argmin.shape, dtype=argmin.dtype).pin_memory()]
    h2d = sum(t.numel() * t.element_size() for t in h_in)
    d2h = sum(t.numel() * t.element_size() for t in h_out)
    e2e_units = 0
    best = -1
    torch.cuda.synchronize(dev)
    te = time.perf_counter()
    for _ in range(Ke):
        mmpc.mmpc_step_host(solver.ctx, meta, h_in[0], h_in[1] if m else None, h_in[2], h_out[0], h_out[2], h_out[3],
                            h_out[1], stream)
        best = int(h_out[3][0])  # the step's result, read on the host
    e2e_ms = (time.perf_counter() - te) * 1e3 / Ke
    e2e_units = int((h_out[1][:, :3].max(dim=1).values <= TOL).sum()) * Ke
    e2e_conv = e2e_units / Ke
    agg = combine_ranks(dict(units=B, ms=ms, e2e_units=B, e2e_ms=e2e_ms), world, dist)
    conv_agg = combine_ranks(dict(units=units_per_step, ms=ms, e2e_units=e2e_conv, e2e_ms=e2e_ms), world, dist)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    N = params["N"]
    passes = iters_sum + B
    exec_ops = alu_ops(N, n, passes, elements)
    ops = alu_ops(N, n, passes, passes * N * m)  # the algorithm's work: every obstacle-sample pair
    achieved = ops / (solve_avg * 1e-3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    sfu_ops = elements
    out = {
        "metric": METRIC,
        "value": agg["units"] / (agg["ms"] * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": agg["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(params, B, m), "goals_per_scene": B, "obstacles": m,
                   "culling": bool(params["cull"]), "kernel_variant": params["variant"],
                   "samples": N, "coefficients": n, "max_iters": params["iters"], "tol_m": TOL,
                   "check_every": CHECK_EVERY, "scenes_per_gpu": 1, "start": "cold",
                   "stall_stop": list(STALL) if args.stall else None,
                   "l2": "flushed between timed steps (256 MiB memset outside the event brackets)"},
        "roofline": {"bound": "alu", "kernel": "am_solve_kernel", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s (FP32 lane ops)", "frac": achieved / peak,
                     "traffic": (measured_traffic("am_solve_kernel", workload_name(params, B, m))
                                 if params["cull"] and params["variant"] == 0 and not args.stall else None),
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                     "peak_basis": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ:.0f} MHz",
                     "ops_per_launch": ops, "launch_ms": solve_avg,
                     "ops_basis": "per trajectory-iteration 14 N n + 7 n^2 (basis and QP products) + 10 m N "
                                  "(obstacle projections) + 60 N (element-wise); culled obstacle-sample pairs "
                                  "are exact zeros, so this is the algorithm's work whether or not the kernel "
                                  "skips them",
                     "evaluated_pairs_per_launch": elements, "dense_pairs_per_launch": passes * N * m,
                     "executed_ops_per_launch": exec_ops,
                     "executed_achieved": exec_ops / (solve_avg * 1e-3) / 1e12,
                     "executed_frac": exec_ops / (solve_avg * 1e-3) / 1e12 / peak,
                     "sfu_frac": sfu_ops / (solve_avg * 1e-3) / (SM_COUNT * SFU_PER_SM * SM_MAX_MHZ * 1e6)},
        "e2e": {"value": agg["e2e_units"] / (agg["e2e_ms"] * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": agg["e2e_ms"], "steps": Ke,
                "api": "mmpc_step_host (one C-ABI call per step, pinned host buffers)", "best_goal": best},
        "gpu_launches": 2 * K,
        "clocks": clocks,
        "detail": {"converged_per_step": conv_agg["units"], "trajectories_per_step": B * world,
                   "converged_fraction": conv_agg["units"] / (B * world),
                   "converged_per_s": conv_agg["units"] / (agg["ms"] * 1e-3),
                   "mpc_solves_per_s": world / (agg["ms"] * 1e-3), "iterations_run": iters_sum,
                   "solve_ms": solve_avg, "score_ms": ms - solve_avg, "wall_s": wall,
                   "step_ms_p50": statistics.median(step_ms), "step_ms_max": max(step_ms)},
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sc, params, sample_stride=max(4, B // 256))
    solver.close()
    if dist is not None:
        dist.destroy_process_group()
    return out


BATCH_SCENES = 256


def batch_workload(seed: int, S: int = BATCH_SCENES):
    """The batching workload: S independent highway scenes with goals
    B ~ U{16..512}, obstacles m ~ U{5..40}, N in {50, 100, 150}."""
    from paper_2109_10392_gb300 import scenes
    scs = scenes.scene_batch(seed, S=S)
    out = []
    for sc in scs:
        p = dict(sc.params)
        p.update(tol=TOL, check_every=CHECK_EVERY)
        out.append((sc, p))
    return out


def run_batch(args):
    """One step = one replay of a CUDA graph holding mmpc_batch_run over all
    scenes (reset, persistent solve, score, per-scene argmin)."""
    import torch

    from paper_2109_10392_gb300 import mmpc

    rank, world, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    work = batch_workload(seed=rank)
    S = len(work)
    # all inputs in one flat device buffer (one host->device copy per step)
    pieces, views = [], []
    off = 0
    if args.stall:
        for _, p in work:
            p.update(stall_tol=STALL[0], stall_ratio=STALL[1])
    for sc, _ in work:
        shapes = [(4,), (sc.obst.shape[0], 4), (len(sc.goals), 3)]
        arrs = [sc.ego, sc.obst.reshape(-1, 4), sc.goals]
        v = []
        for a, shp in zip(arrs, shapes):
            k = int(np.prod(shp))
            pieces.append(np.asarray(a, dtype=np.float32).ravel())
            v.append((off, k, shp))
            off += k
        views.append(v)
    h_in = torch.from_numpy(np.concatenate(pieces)).pin_memory()
    d_in = torch.empty(h_in.shape, dtype=torch.float32, device=dev)
    d_in.copy_(h_in)
    descs = []
    for (sc, p), v in zip(work, views):
        ts = [d_in[o:o + k].view(*shp) for o, k, shp in v]
        descs.append(dict(params=p, ego=ts[0], obst=ts[1] if sc.obst.shape[0] else None, goals=ts[2]))
    meta = mmpc.make_meta(**work[0][0].meta)
    t_setup = time.perf_counter()
    bt = mmpc.Batch(descs, meta)
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        schedule = bt.autotune() if args.schedule == 0 else (bt.set_schedule(args.schedule) or args.schedule)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        bt.run()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            graph.replay()
    torch.cuda.synchronize(dev)
    Btot = sum(len(sc.goals) for sc, _ in work)
    resid = bt.flat["resid"].view(-1, 4)
    conv = int((resid[:, :3].max(dim=1).values <= TOL).sum().item())
    iters_all = bt.flat["iters"].to(torch.int64).cpu().numpy()
    # scene-by-scene latencies: completion time of each scene since the first
    # CTA of the launch started (every scene is submitted at launch)
    lat = []
    with torch.cuda.stream(stream):
        for _ in range(max(3, min(20, args.steps))):
            flush.zero_()
            graph.replay()
            ms_s, _ = bt.times()
            lat.append(ms_s.copy())
    lat = np.concatenate(lat)
    bt.take_work_count()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(K):
            flush.zero_()
            ev[i][0].record(stream)
            graph.replay()
            ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    elements = bt.take_work_count() / K
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    ms = sum(step_ms) / K

    # end to end: inputs copied from pinned host memory, the graph replayed,
    # coefficients, costs and argmins copied back
    Ke = min(K, args.e2e_steps)
    outs = [bt.flat["coef"], bt.flat["cost"], bt.flat["argmin"]]
    h_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
    h2d = h_in.numel() * 4
    d2h = sum(t.numel() * t.element_size() for t in h_out)
    torch.cuda.synchronize(dev)
    te = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(Ke):
            d_in.copy_(h_in, non_blocking=True)
            graph.replay()
            for h, d in zip(h_out, outs):
                h.copy_(d, non_blocking=True)
            stream.synchronize()
    e2e_ms = (time.perf_counter() - te) * 1e3 / Ke
    agg = combine_ranks(dict(units=Btot, ms=ms, e2e_units=Btot, e2e_ms=e2e_ms), world, dist)
    sagg = combine_ranks(dict(units=S, ms=ms, e2e_units=S, e2e_ms=e2e_ms), world, dist)
    if rank != 0:
        bt.close()
        if dist is not None:
            dist.destroy_process_group()
        return None

    # dense algorithmic work, summed over scenes (as for one scene)
    ops = 0.0
    for i, (sc, p) in enumerate(work):
        oc, ob = bt.offsets[i]
        B, m, N, n = len(sc.goals), sc.obst.shape[0], p["N"], p["n"]
        passes = int(iters_all[ob:ob + B].sum()) + B
        ops += alu_ops(N, n, passes, passes * N * m)
    achieved = ops / (ms * 1e-3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    Ns = sorted({p["N"] for _, p in work})
    out = {
        "metric": METRIC,
        "value": agg["units"] / (agg["ms"] * 1e-3),
        "unit": UNIT,
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": agg["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"highway_batch_S{S}_B16-512_m5-40_N{'-'.join(map(str, Ns))}_n12_K100_tol{TOL:g}",
                   "scenes_per_gpu": S, "trajectories_per_gpu": Btot, "schedule": schedule,
                   "launch_shapes": bt.describe()["launches"],
                   "stall_stop": list(STALL) if args.stall else None,
                   "graph": "one CUDA graph replay per step", "start": "cold",
                   "l2": "flushed between timed steps (256 MiB memset outside the event brackets)"},
        "roofline": {"bound": "alu", "kernel": "am_solve_batch_kernel", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s (FP32 lane ops)", "frac": achieved / peak,
                     "traffic": (measured_traffic("am_solve_batch_kernel", f"highway_batch_S{S}_B16-512_m5-40_N"
                                                  f"{'-'.join(map(str, Ns))}_n12_K100_tol{TOL:g}")
                                 if schedule == 4 and not args.stall else None),
                     "traffic_unit": "bytes per step (ncu dram__bytes_read.sum + dram__bytes_write.sum over the "
                                     "three horizon-group launches)",
                     "peak_basis": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ:.0f} MHz",
                     "ops_per_launch": ops, "launch_ms": ms,
                     "ops_basis": "dense algorithmic ops summed over scenes, over the whole graph step (reset, "
                                  "solve, score, argmin kernels)",
                     "evaluated_pairs_per_launch": elements},
        "e2e": {"value": agg["e2e_units"] / (agg["e2e_ms"] * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": agg["e2e_ms"], "steps": Ke,
                "mpc_solves_per_s": sagg["e2e_units"] / (sagg["e2e_ms"] * 1e-3)},
        "gpu_launches": 4 * K,
        "clocks": clocks,
        "detail": {"mpc_solves_per_s": sagg["units"] / (sagg["ms"] * 1e-3),
                   "scene_latency_ms_p50": float(np.percentile(lat, 50)),
                   "scene_latency_ms_p99": float(np.percentile(lat, 99)),
                   "scene_latency_ms_max": float(lat.max()),
                   "converged_fraction": conv / Btot, "iterations_run": int(iters_all.sum()),
                   "setup_s": setup_s, "wall_s": wall,
                   "step_ms_p50": statistics.median(step_ms), "step_ms_max": max(step_ms)},
    }
    bt.close()
    if dist is not None:
        dist.destroy_process_group()
    return out


HEADLINE = "warm_fallback"  # the target form: batched, learned warm start, cold fallback of every miss, stall stop


def _warm_ops(N, n, m, passes):
    """Dense algorithmic lane operations of `passes` AM passes (alu_ops)."""
    return alu_ops(N, n, passes, passes * N * m)


def run_warm(args):
    """The metric: trajectories/s that reach residual <= 1e-2 m on fresh dense
    highway scenes (4096 scenes x 256 goals, 50 obstacles), for the
    warm-started, batched form (the network trained here, on the GPU, by the
    library's kernels; cold fallback of the misses; opt-in stall stop)
    against the plain cold-started GPU method on the same scenes.  One step =
    one CUDA graph replay over all evaluation scenes (features, network,
    decode, persistent solve, fallback solve, score)."""
    import torch

    from paper_2109_10392_gb300 import mmpc, warmstart

    rank, world, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    cfg = warmstart.WarmConfig(train_scenes=args.warm_train_scenes, steps=args.warm_steps, seed=rank)
    t0 = time.perf_counter()
    X, T = warmstart.build_dataset(cfg, dev)
    t1 = time.perf_counter()
    ws, losses = warmstart.train(cfg, X, T, dev)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    Xv, Tv = warmstart.build_dataset(cfg, dev, seed_offset=7_777_777, S=max(256, cfg.train_scenes // 50))
    val = warmstart.validation_loss(ws, Xv, Tv)
    train_rows = int(X.shape[0])
    del X, T, Xv, Tv
    S, B = args.warm_eval_scenes, 256
    seed = 10**6 + rank
    fwd = warmstart.time_forward(ws, S * B, dev)
    reps = 3
    from paper_2109_10392_gb300 import mmpc as _m
    dense = warmstart.evaluate(ws, cfg, dev, S=S, B=B, reps=reps, seed=seed, plain=True)
    ev32 = warmstart.evaluate(ws, cfg, dev, S=S, B=B, reps=reps, seed=seed, stall=STALL)
    evbf = warmstart.evaluate(ws, cfg, dev, S=S, B=B, reps=reps, seed=seed, stall=STALL,
                              precision=_m.MMPC_PREC_BF16_SPLIT)
    # the target form: tensor-core solves in TF32 hi + lo (FP32-class positions)
    ev = warmstart.evaluate(ws, cfg, dev, S=S, B=B, reps=reps, seed=seed, stall=STALL, keep=True,
                            precision=_m.MMPC_PREC_TF32_SPLIT)
    keep = ev.pop("_keep")
    plain = dense["plain"]
    for e_ in (ev, ev32, evbf):
        for k in ("cold", "warm", "warm_fallback", "warm_fallback_budget", "warm_fallback_near"):
            e_[f"{k}_vs_plain"] = e_[k]["trajectories_per_s"] / plain["trajectories_per_s"]
            e_[f"{k}_converged_vs_plain"] = e_[k]["converged_per_s"] / plain["converged_per_s"]
            e_[f"{k}_converged_vs_batched_cold"] = e_[k]["converged_per_s"] / dense["cold"]["converged_per_s"]
            e_[f"{k}_converged_vs_batched_cold_stall"] = e_[k]["converged_per_s"] / ev32["cold"]["converged_per_s"]
            # against the batched cold start on the same kernel, with the stall stop
            e_[f"{k}_converged_vs_same_kernel_cold"] = e_[k]["converged_per_s"] / e_["cold"]["converged_per_s"]
    warm, stream = keep["warm"], keep["stream"]
    graph = keep["graphs"][HEADLINE]
    converged = ev[HEADLINE]["converged"]

    # the headline: K replays of the target form's graph between L2-sized
    # input sets (the 1M-trajectory outputs alone exceed L2), CUDA events on
    # the replay stream, clocks sampled meanwhile
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
    torch.cuda.synchronize(dev)
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    tw = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler capture the timed region alone
    with torch.cuda.stream(stream):
        for i in range(K):
            evs[i][0].record(stream)
            graph.replay()
            evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_pop()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - tw
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / K
    conv_now = int((warm.flat["resid"].view(-1, 4)[:, :3].max(dim=1).values <= TOL).sum().item())

    # the dominant kernel: am_solve_batch_kernel (the warm solve and the
    # fallback solve of each step), timed by events the library records on
    # the run's stream around the two launches, in eager runs of the same step
    p = cfg.params
    N, n, m = int(p["N"]), int(p["n"]), cfg.obstacles
    tev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in tev:  # torch creates the CUDA event at its first record
        e.record(stream)
    torch.cuda.synchronize(dev)
    warm.set_fallback(1)
    warm.set_timing(tev)
    warm.take_work_count()
    solve_ms, fb_ms, R = 0.0, 0.0, 3
    for _ in range(R):
        with torch.cuda.stream(stream):
            keep["step"]()
        torch.cuda.synchronize(dev)
        solve_ms += tev[0].elapsed_time(tev[1]) / R
        fb_ms += tev[2].elapsed_time(tev[3]) / R
    warm.set_timing(None)
    elements = warm.take_work_count() / R
    passes = ev[HEADLINE]["passes"]
    launch_ms = (solve_ms + fb_ms) / 2
    # am_solve_tc_kernel (both launches of a step): the basis products on the
    # tensor cores, the rest -- projections, element-wise work, QP products --
    # on the FP32 pipes, which bound it (issue-bound; the tensor pipe is a few
    # percent busy).  ALU roofline over the FP32-pipe part of the count; the
    # tensor part against the TF32 peak beside it.
    alu = passes * (7 * n * n + 60 * N) + OPS_PER_ELEMENT * passes * N * m
    alu_exec = passes * (7 * n * n + 60 * N) + OPS_PER_ELEMENT * elements
    ops = _warm_ops(N, n, m, passes)  # the per-unit count of every AM pass (both launches)
    achieved = ops / 2 / (launch_ms * 1e-3) / 1e12
    peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    mma_flops = 2.0 * 14 * N * n * passes  # the algorithm's basis products, as tensor FLOPs
    tf32_peak = tensor_peak_tflops("tf32")
    traffic = measured_traffic("am_solve_tc_kernel", f"highway_warm_S{S}_B{B}_m{m}_N{N}_n{n}")

    # end to end through the library's public calls with host buffers: the
    # step's inputs copied in from pinned memory, the graph replayed, every
    # output (coefficients, residuals, iterations, costs, per-scene argmin)
    # copied back, the stream synchronised
    ins = keep["inputs"]
    h_in = {k: v.cpu().pin_memory() for k, v in ins.items()}
    outs = [warm.flat[k] for k in ("coef", "resid", "iters", "cost", "argmin")]
    h_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
    h2d = sum(t.numel() * t.element_size() for t in h_in.values())
    d2h = sum(t.numel() * t.element_size() for t in h_out)
    Ke = max(1, min(K, args.e2e_steps))
    e2e_conv = 0
    torch.cuda.synchronize(dev)
    te = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(Ke):
            for k, v in ins.items():
                v.copy_(h_in[k], non_blocking=True)
            graph.replay()
            for h, d in zip(h_out, outs):
                h.copy_(d, non_blocking=True)
            stream.synchronize()
            e2e_conv = int((h_out[1][:, :3].max(dim=1).values <= TOL).sum())
    e2e_ms = (time.perf_counter() - te) * 1e3 / Ke

    # the library's launches per step: features; the network's forward (one
    # launch of the single-kernel network); decode; the batch run (reset,
    # order, solve, fallback compaction, fallback solve, score, finish)
    launches_per_step = 1 + ws.net.forward_launches(S * B) + 1 + 7
    agg = combine_ranks(dict(units=converged, ms=ms, e2e_units=e2e_conv, e2e_ms=e2e_ms), world, dist)
    tagg = combine_ranks(dict(units=S * B, ms=ms, e2e_units=S * B, e2e_ms=e2e_ms), world, dist)
    if rank != 0:
        keep["warm"].close()
        keep["cold"].close()
        ws.close()
        if dist is not None:
            dist.destroy_process_group()
        return None

    sparse = warmstart.evaluate(ws, cfg, dev, S=S, B=B, reps=reps, seed=2 * 10**6 + rank,
                                obstacles=10, x_range=(-30.0, 120.0))
    ws.close()
    scene = _scene_throughput(dev)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_warm(p, S, B, m, cfg.x_range, seed)
    out = {
        "metric": METRIC, "value": agg["units"] / (agg["ms"] * 1e-3), "unit": UNIT_CONV, "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": agg["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "tf32 hi+lo (tensor) + f32", "data": "synthetic",
        "config": {"workload": f"highway_warm_S{S}_B{B}_m{m}_N{N}_n{n}_K{p['iters']}_tol{TOL:g}",
                   "form": "batched (one persistent tensor-core launch over all scenes), learned warm start "
                           "(lambda0 = Q c0), cold fallback of every miss, stall stop (residual > 1 m and not "
                           "halved over two checks); basis products TF32 hi + lo on tcgen05 with FP32 "
                           "accumulation, projections and QP steps FP32", "scenes_per_gpu": S, "goals_per_scene": B,
                   "obstacles": m,
                   "samples": N, "coefficients": n, "max_iters": int(p["iters"]), "tol_m": TOL,
                   "check_every": CHECK_EVERY, "stall_stop": list(STALL),
                   "train_scenes": cfg.train_scenes, "train_rows": train_rows, "train_steps": cfg.steps,
                   "network": list(cfg.widths), "graph": "one CUDA graph replay per step",
                   "l2": "inputs larger than L2: each step reads 4096 scenes and writes 1M trajectories' "
                         "outputs (>150 MB)"},
        "roofline": {"bound": "alu", "kernel": "am_solve_tc_kernel", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s (FP32 lane ops)", "frac": achieved / peak, "traffic": traffic,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum), "
                                     "null when not measured for this kernel source",
                     "peak_basis": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ:.0f} MHz",
                     "ops_basis": "per trajectory-iteration 14 N n (basis products, here on the tensor cores) + "
                                  "7 n^2 (QP products) + 10 m N (obstacle projections) + 60 N (element-wise), over "
                                  "every AM pass the two launches of a step ran (warm solve, cold fallback)",
                     "ops_per_launch": ops / 2, "launch_ms": launch_ms, "launches_per_step": 2,
                     "solve_launch_ms": solve_ms, "fallback_launch_ms": fb_ms,
                     "fp32_pipe_part": {"ops_per_launch": alu / 2,
                                        "achieved": alu / 2 / (launch_ms * 1e-3) / 1e12,
                                        "frac": alu / 2 / (launch_ms * 1e-3) / 1e12 / peak,
                                        "basis": "the count without the 14 N n basis products (the work the FP32 "
                                                 "pipes carry)"},
                     "evaluated_pairs_per_step": elements, "dense_pairs_per_step": passes * N * m,
                     "executed_ops_per_launch": alu_exec / 2,
                     "executed_frac": alu_exec / 2 / (launch_ms * 1e-3) / 1e12 / peak,
                     "tensor": {"achieved": mma_flops / 2 / (launch_ms * 1e-3) / 1e12, "peak": tf32_peak,
                                "unit": "TFLOP/s", "frac": mma_flops / 2 / (launch_ms * 1e-3) / 1e12 / tf32_peak,
                                "basis": "2 x 14 N n FLOPs per trajectory-iteration (the algorithm's basis "
                                         "products; the hi + lo split issues three times as many) against the "
                                         "TF32 dense peak = measured BF16 burst x 1.1 / 2.25 (nominal ratio)"}},
        "e2e": {"value": agg["e2e_units"] / (agg["e2e_ms"] * 1e-3), "unit": UNIT_CONV,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": agg["e2e_ms"], "steps": Ke,
                "trajectories_per_s": tagg["e2e_units"] / (tagg["e2e_ms"] * 1e-3),
                "api": "inputs copied from pinned host memory, the step's CUDA graph (features, network, decode, "
                       "mmpc_batch_run) replayed, all outputs copied back, stream synchronised"},
        "gpu_launches": launches_per_step * K,
        "clocks": clocks,
        "detail": {"converged_per_step": converged, "converged_in_timed_steps": conv_now,
                   "trajectories_per_step": S * B, "trajectories_per_s": tagg["units"] / (tagg["ms"] * 1e-3),
                   "mpc_solves_per_s": S * world / (agg["ms"] * 1e-3),
                   "plain_converged_per_s": plain["converged_per_s"],
                   "ratio_vs_plain": ev[HEADLINE]["converged_per_s"] / plain["converged_per_s"],
                   "ratio_vs_batched_cold": ev[HEADLINE]["converged_per_s"] / dense["cold"]["converged_per_s"],
                   "ratio_vs_batched_cold_stall": ev[HEADLINE]["converged_per_s"] / ev32["cold"]["converged_per_s"],
                   "variants_no_stall": dense, "variants_stall_stop_tensor_tf32x2": ev,
                   "variants_stall_stop_fp32": ev32, "variants_stall_stop_tensor_bf16x2": evbf,
                   "sparse_10_obstacles": sparse,
                   "scene_1024_goals_plain_cold": scene, "val_loss": val, "network_forward": fwd,
                   "loss_first_last": [losses[0][1], losses[-1][1]], "dataset_s": t1 - t0, "train_s": t2 - t1,
                   "train_step_ms": ws.train_step_ms, "train_tensor_cores": cfg.tensor_training,
                   "wall_s": wall, "step_ms_p50": statistics.median(step_ms), "step_ms_max": max(step_ms)},
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    keep["warm"].close()
    keep["cold"].close()
    if dist is not None:
        dist.destroy_process_group()
    return out


def _scene_throughput(dev, target_s=0.5):
    """Plain cold-started solve + score of the 1024-goal, 50-obstacle scene
    (N = 100, n = 12, 100 iterations, residual target 1e-2 m), CUDA events
    between L2 flushes, about target_s of steps."""
    import torch

    from paper_2109_10392_gb300 import mmpc
    sc, params = workload(seed=0, kind="scene")
    B, m, n = len(sc.goals), sc.obst.shape[0], params["n"]
    solver = mmpc.Solver(params, m)
    meta = mmpc.make_meta(**sc.meta)
    f32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev).contiguous()  # noqa: E731
    ego, obst, goals = f32(sc.ego), f32(sc.obst), f32(sc.goals)
    coef = torch.empty((B, 3 * n), device=dev)
    resid = torch.empty((B, 4), device=dev)
    iters = torch.empty((B,), dtype=torch.int32, device=dev)
    cost = torch.empty((B,), device=dev)
    am = torch.empty((1,), dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    ms = []
    for i in range(5 + int(target_s / 4e-4)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mmpc.mmpc_solve(solver.ctx, ego, obst, goals, coef, None, None, None, resid, iters, stream)
        mmpc.mmpc_score(solver.ctx, meta, coef, cost, am, stream)
        b.record(stream)
        if i >= 5:
            ms.append((a, b))
    torch.cuda.synchronize(dev)
    solver.status()
    t = [a.elapsed_time(b) for a, b in ms]
    conv = int((resid[:, :3].max(dim=1).values <= TOL).sum().item())
    solver.close()
    avg = sum(t) / len(t)
    return dict(workload=workload_name(params, B, m), steps=len(t), ms_per_step=avg, trajectories_per_s=B / (avg * 1e-3),
                converged=conv, converged_per_s=conv / (avg * 1e-3))


def _oracle_run(sc, params, idx, threads):
    import oracle
    p = oracle.params(**params)
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    t0 = time.perf_counter()
    r = oracle.solve(p, f(sc.ego), f(sc.obst), f(sc.goals)[idx], nthreads=threads)
    dt = time.perf_counter() - t0
    conv = int((r["resid"][:, :3].max(axis=1) <= TOL).sum())
    return dt, conv


def cpu_baseline(sc, params, sample_stride=4, single_sample=16):
    """The FP64 oracle, as it stands, on the host cores, on every
    `sample_stride`-th goal of the same scene (all cores, OpenMP over
    trajectories), and on `single_sample` of those goals single-threaded."""
    threads = os.cpu_count() or 1
    idx = np.arange(0, len(sc.goals), sample_stride)
    dt, conv = _oracle_run(sc, params, idx, threads)
    dt1, _ = _oracle_run(sc, params, idx[:single_sample], 1)
    return {"value": len(idx) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(idx)} of {len(sc.goals)} goals (every {sample_stride}th), same scene and stopping rule",
            "converged_fraction": conv / len(idx), "seconds": dt,
            "single_thread": {"value": min(single_sample, len(idx)) / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"the first {min(single_sample, len(idx))} goals of that sample"}}


def _warm_eval_scenes(params, S, B, m, x_range, seed):
    """The evaluation scenes of the warm workload as the GPU receives them
    (the same seeded stack, rounded to float32), scene-major."""
    from paper_2109_10392_gb300 import scenes
    ego, obst, goals = scenes.scene_stack(seed, S, B, m, x_range, goals="grid" if B % 8 == 0 else "random")
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    return f(ego), f(obst), f(goals)


def _oracle_scenes(params, ego, obst, goals, idx, threads):
    """The FP64 oracle, cold start, on scenes idx (all goals of each, OpenMP
    over goals); returns (seconds, trajectories, converged)."""
    import oracle
    p = oracle.params(**dict(params, tol=TOL, check_every=CHECK_EVERY))
    t0 = time.perf_counter()
    units = conv = 0
    for i in idx:
        r = oracle.solve(p, ego[i], obst[i], goals[i], nthreads=threads)
        units += goals.shape[1]
        conv += int((r["resid"][:, :3].max(axis=1) <= TOL).sum())
    return time.perf_counter() - t0, units, conv


def cpu_baseline_warm(params, S, B, m, x_range, seed, budget_s=15.0):
    """The FP64 oracle as it stands (the plain cold-started method) on the
    host cores, on the first evaluation scenes of the warm workload, as many
    as fit in about budget_s; converged trajectories per second."""
    threads = os.cpu_count() or 1
    ego, obst, goals = _warm_eval_scenes(params, S, B, m, x_range, seed)
    dt1, _, _ = _oracle_scenes(params, ego, obst, goals, [0], threads)
    k = int(max(1, min(S, budget_s / max(dt1, 1e-3))))
    dt, units, conv = _oracle_scenes(params, ego, obst, goals, range(k), threads)
    return {"value": conv / dt, "unit": UNIT_CONV, "cores": threads, "kind": "oracle",
            "sample": f"the first {k} of the {S} evaluation scenes, all {B} goals each ({units} trajectories), "
                      "cold start, same stopping rule", "trajectories_per_s": units / dt, "converged": conv,
            "seconds": dt}


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return None
    threads = os.cpu_count() or 1
    if args.workload != "warm":
        return run_reference_scene(args)
    from paper_2109_10392_gb300 import warmstart
    cfg = warmstart.WarmConfig(seed=0)
    p = cfg.params
    S, B, m = args.warm_eval_scenes, 256, cfg.obstacles
    ego, obst, goals = _warm_eval_scenes(p, S, B, m, cfg.x_range, 10**6)
    # size one step so that warmup + steps take about a minute in total
    dt1, _, _ = _oracle_scenes(p, ego, obst, goals, [0], threads)
    per_step = 60.0 / max(1, args.steps + args.warmup)
    k = int(max(1, min(S // max(1, args.steps + args.warmup), per_step / max(dt1, 1e-3))))
    pos = 1
    for _ in range(args.warmup):
        _oracle_scenes(p, ego, obst, goals, range(pos, pos + k), threads)
        pos += k
    units = conv = 0
    secs = 0.0
    for _ in range(args.steps):
        dt, u, c = _oracle_scenes(p, ego, obst, goals, range(pos, pos + k), threads)
        pos += k
        units += u
        conv += c
        secs += dt
    value = conv / secs
    return {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT_CONV, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"highway_warm_S{S}_B{B}_m{m}_N{p['N']}_n{p['n']}_K{p['iters']}_tol{TOL:g}",
                   "form": "the FP64 oracle (plain method, cold start) on consecutive evaluation scenes",
                   "scenes_per_step": k, "trajectories_per_step": k * B},
        "cpu_baseline": {"value": value, "unit": UNIT_CONV, "cores": threads, "kind": "oracle",
                         "sample": f"{k} evaluation scenes x {B} goals per step, cold start, same stopping rule",
                         "trajectories_per_s": units / secs, "converged": conv},
        "e2e": {"value": value, "unit": UNIT_CONV, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def run_reference_scene(args):
    """The oracle on a bounded sample of the 1024-goal scene per step (the
    reference arm of the single-scene workloads)."""
    sc, params = workload(seed=0)
    threads = os.cpu_count() or 1
    # size one step so that warmup + steps take about a minute in total
    t1, _ = _oracle_run(sc, params, np.array([0]), 1)
    per_step = 60.0 / max(1, args.steps + args.warmup)
    ntraj = int(max(1, min(len(sc.goals), math.floor(per_step * threads / max(t1, 1e-6)))))
    stride = max(1, len(sc.goals) // ntraj)
    rng_off = 0
    for _ in range(args.warmup):
        _oracle_run(sc, params, np.arange(rng_off % stride, len(sc.goals), stride)[:ntraj], threads)
    units, secs, conv_all = 0, 0.0, 0
    for i in range(args.steps):
        idx = np.arange(i % stride, len(sc.goals), stride)[:ntraj]
        dt, conv = _oracle_run(sc, params, idx, threads)
        units += len(idx)
        conv_all += conv
        secs += dt
    value = units / secs
    return {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(params, len(sc.goals), sc.obst.shape[0]),
                   "trajectories_per_step": ntraj},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{ntraj} of {len(sc.goals)} goals per step (strided), same scene and stopping rule",
                         "converged_fraction": conv_all / max(1, units)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


PRECISION_MODES = ((0, 0, "fp32 (CUDA cores)"), (3, 1, "tf32 (tensor)"), (3, 2, "tf32 hi+lo (tensor)"),
                   (3, 3, "bf16 (tensor)"), (3, 4, "bf16 hi+lo (tensor)"))


def run_precision(args):
    """The precision workload (16384 goals, 30 obstacles, N = 200, n = 16):
    solve + score per step under the metric's stopping rule, for the FP32
    kernel and the tensor-core kernel in each precision; the headline is the
    tensor-core TF32 hi + lo mode.  The error of each mode against the FP64
    oracle is measured by the GPU tests, not here."""
    import torch

    from paper_2109_10392_gb300 import mmpc
    rank, world, _ = rank_env()
    if world > 1:
        raise SystemExit("--workload precision runs on one GPU")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sc, params = workload(seed=0, kind="precision")
    B, m, n, N = len(sc.goals), sc.obst.shape[0], params["n"], params["N"]
    f32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev).contiguous()  # noqa: E731
    ego, obst, goals = f32(sc.ego), f32(sc.obst), f32(sc.goals)
    meta = mmpc.make_meta(**sc.meta)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows, coefs = {}, {}
    sampler = ClockSampler(0)
    sampler.start()
    for variant, prec, name in PRECISION_MODES:
        p = dict(params, variant=variant, precision=prec)
        solver = mmpc.Solver(p, m)
        coef = torch.empty((B, 3 * n), device=dev)
        resid = torch.empty((B, 4), device=dev)
        iters = torch.empty((B,), dtype=torch.int32, device=dev)
        cost = torch.empty((B,), device=dev)
        am = torch.empty((1,), dtype=torch.int32, device=dev)

        def step():
            mmpc.mmpc_solve(solver.ctx, ego, obst, goals, coef, None, None, None, resid, iters, stream)
            mmpc.mmpc_score(solver.ctx, meta, coef, cost, am, stream)

        for _ in range(args.warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize(dev)
        solver.status()
        ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
        conv = int((resid[:, :3].max(dim=1).values <= TOL).sum().item())
        rows[name] = dict(ms_per_step=ms, trajectories_per_s=B / (ms * 1e-3), converged=conv,
                          converged_per_s=conv / (ms * 1e-3), mean_iters=float(iters.double().mean().item()),
                          argmin=int(am.item()))
        coefs[name] = (coef.double().cpu().numpy(), cost.double().cpu().numpy())
        solver.close()
    clocks = sampler.stop()
    head = rows["tf32 hi+lo (tensor)"]
    return {
        "metric": METRIC, "value": head["converged_per_s"], "unit": UNIT_CONV, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "tf32 hi+lo (tensor) + f32", "data": "synthetic",
        "config": {"workload": workload_name(params, B, m), "goals_per_scene": B, "obstacles": m, "samples": N,
                   "coefficients": n, "max_iters": params["iters"], "tol_m": TOL, "check_every": CHECK_EVERY,
                   "l2": "flushed between timed steps (256 MiB memset outside the event brackets)",
                   "form": "tensor-core kernel (variant 3), TF32 hi + lo basis products; the other modes in detail"},
        "clocks": clocks,
        "detail": {"modes": rows,
                   "error_vs_fp64_oracle": "tests/test_gpu_tensorcore.py::test_precision_workload_error_table",
                   "speedup_tf32x2_vs_fp32": rows["fp32 (CUDA cores)"]["ms_per_step"] / head["ms_per_step"]},
    }


SWEEP_B = (11, 32, 128, 512, 1024, 2048, 4096, 16384, 65536)


def run_sweep(args):
    """Trajectories/s against the batch size (the counterpart of the paper's
    time-vs-batch-size experiment, Fig. 2b): one dense scene of the
    1024-goal distribution (50 obstacles, N = 100, n = 12, 100 iterations,
    residual target 1e-2 m) per B, solve + score timed with CUDA events
    between L2 flushes; and one MPC cycle of the paper's own setting (11 goals,
    10 obstacles), the figure its Table V times on a CPU."""
    import torch

    from paper_2109_10392_gb300 import mmpc, scenes
    rank, world, _ = rank_env()
    if world > 1:
        raise SystemExit("--workload sweep runs on one GPU")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    f32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev).contiguous()  # noqa: E731

    def time_scene(sc, target_s=0.5):
        params = dict(sc.params, tol=TOL, check_every=CHECK_EVERY)
        B, m, n = len(sc.goals), sc.obst.shape[0], params["n"]
        solver = mmpc.Solver(params, m)
        meta = mmpc.make_meta(**sc.meta)
        ego, obst, goals = f32(sc.ego), f32(sc.obst), f32(sc.goals)
        coef = torch.empty((B, 3 * n), dtype=torch.float32, device=dev)
        resid = torch.empty((B, 4), dtype=torch.float32, device=dev)
        iters = torch.empty((B,), dtype=torch.int32, device=dev)
        cost = torch.empty((B,), dtype=torch.float32, device=dev)
        argmin = torch.empty((1,), dtype=torch.int32, device=dev)

        def step(e0=None, e1=None):
            flush.zero_()
            if e0 is not None:
                e0.record(stream)
            mmpc.mmpc_solve(solver.ctx, ego, obst, goals, coef, None, None, None, resid, iters, stream)
            mmpc.mmpc_score(solver.ctx, meta, coef, cost, argmin, stream)
            if e1 is not None:
                e1.record(stream)

        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            step(a, b)
        torch.cuda.synchronize(dev)
        est = max(a.elapsed_time(b), 1e-3)
        K = int(min(2000, max(5, target_s * 1e3 / est)))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for e0, e1 in ev:
            step(e0, e1)
        torch.cuda.synchronize(dev)
        solver.status()
        ms = sorted(e0.elapsed_time(e1) for e0, e1 in ev)
        conv = int((resid[:, :3].max(dim=1).values <= TOL).sum().item())
        solver.close()
        return dict(B=B, obstacles=m, steps=K, ms_median=ms[K // 2], ms_mean=sum(ms) / K,
                    trajectories_per_s=B / (sum(ms) / K * 1e-3), us_per_trajectory=sum(ms) / K * 1e3 / B,
                    converged=conv)

    sampler = ClockSampler(0)
    sampler.start()
    curve = [time_scene(scenes.scene_custom(seed=B, B=B, m=50, N=100, n=12)) for B in SWEEP_B]
    cycle = time_scene(scenes.scene_small(0))
    clocks = sampler.stop()
    best = max(curve, key=lambda r: r["trajectories_per_s"])
    return {
        "metric": "trajectories/s against the batch size (one scene per solve)", "value": best["trajectories_per_s"],
        "unit": UNIT, "n_gpus": 1, "steps": None, "warmup": args.warmup, "ms_per_step": best["ms_mean"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "highway_sweep_B11-65536_m50_N100_n12_K100_tol0.01", "sizes": list(SWEEP_B),
                   "l2": "flushed between timed steps (256 MiB memset outside the event brackets)",
                   "timing": "solve + score per step, CUDA events, about 0.5 s of steps per size"},
        "detail": {"curve": curve, "mpc_cycle_paper_setting": cycle,
                   "paper_context": "Table V of the paper: 0.07 s per MPC cycle at batch 11 on an i7-8750 CPU"},
        "clocks": clocks,
    }


def add_measured_peak(roofline: dict) -> None:
    """Beside the derived peak: the FP32 lane-op rate the device reaches on
    saturating FFMA / packed FFMA2 chains (mmpc_measure_peaks, run after the
    timed region), and the fraction of it."""
    from paper_2109_10392_gb300 import mmpc
    pk = mmpc.mmpc_measure_peaks(reps=3)
    lane = max(pk["ffma"], pk["ffma2"]) / 1e12
    roofline["measured_peak"] = {
        "fp32_lane_ops": lane, "ffma": pk["ffma"] / 1e12, "ffma2": pk["ffma2"] / 1e12,
        "rsqrt": pk["rsqrt"] / 1e12, "unit": "T ops/s",
        "lanes_per_sm_per_clk_at_max_clock": lane * 1e12 / (pk["sms"] * pk["clock_khz"] * 1e3),
        "basis": "mmpc_measure_peaks: 8 dependent chains per thread, 64 warps per SM, best of 3"}
    roofline["frac_of_measured"] = roofline["achieved"] / lane


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default per workload: warm 10, scene 2000, precision 20, batch 100; "
                         "--impl reference: 3); a warm step replays the whole 1M-trajectory evaluation")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cull", action="store_true", help="evaluate every obstacle-sample pair (no culling)")
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1, 2],
                    help="solve kernel: 1 one sample per thread, 2 two samples per thread, 0 automatic")
    ap.add_argument("--workload", default="warm", choices=["warm", "scene", "batch", "precision", "sweep"],
                    help="warm (default, the metric): learned warm start (trained in the run), batched, with cold "
                         "fallback and stall stop, against the plain cold-started method on 4096 fresh scenes x "
                         "256 goals; scene: one 1024-goal scene per GPU; batch: 256 uneven scenes per GPU in one "
                         "graph; precision: "
                         "one 16384-goal scene, 30 obstacles, N = 200, n = 16; sweep: trajectories/s against the "
                         "batch size (11 to 65536 goals) and one MPC cycle of the paper's 11-goal setting")
    ap.add_argument("--stall", action="store_true",
                    help="opt-in stall stop (residual > 1 m and not halved over two checks) for scene and batch")
    ap.add_argument("--warm-train-scenes", type=int, default=200_000)
    ap.add_argument("--warm-steps", type=int, default=4000)
    ap.add_argument("--warm-eval-scenes", type=int, default=4096)
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="batch item order (0: autotuned)")
    args = ap.parse_args(argv)
    if args.steps is None:
        args.steps = (3 if args.impl == "reference" else
                      {"precision": 20, "batch": 100, "warm": 10}.get(args.workload, 2000))
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    return args


def main():
    args = parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    else:
        out = {"batch": run_batch, "warm": run_warm, "sweep": run_sweep,
               "precision": run_precision}.get(args.workload, run_mine)(args)
        if out is not None and out.get("roofline", {}).get("bound") == "alu":
            add_measured_peak(out["roofline"])
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
