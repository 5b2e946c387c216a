"""Learned warm start of Algorithm 1: dataset, training, inference, evaluation.

The paper proposes no learned component (it names learning from its batch
solutions as a use of the method, Sec. V).  This module builds one around the
library, every step on the GPU through the C ABI:

* dataset: S seeded highway scenes, a few goals each, solved from the cold
  start by the plain method (Algorithm 1, 100 iterations, Sec. III-E) with
  `mmpc.Batch`; inputs are the feature rows (`mmpc_features`), targets the
  coefficients c of the trajectories that reached the residual target,
  encoded relative to constant-velocity motion and standardised per column
  (`mmpc_warm_encode`, `mmpc_column_stats`).  The multipliers are not
  learned: the warm start takes lambda^0 = Q c^0, the multipliers of a fixed
  point of the iteration (measured: perturbing exact multipliers by 1 % of
  their spread already halves the fraction that converges, while lambda^0 =
  Q c^0 from the exact c converges in one check, 10 iterations);
* training: minibatches gathered on the device (`mmpc_gather_rows`), the
  network's own forward / backward kernels (`mmpc_mlp_loss_grad`) and AdamW
  (`mmpc_mlp_adamw`) with a cosine learning-rate schedule;
* inference: features -> network -> decode (`mmpc_warm_decode`) gives
  (c^0, lambda^0) for `mmpc_solve` / `mmpc.Batch`;
* evaluation: the same scenes solved from the cold start and from the warm
  start, each iterated until its residual is <= tol (checked every 10
  iterations) or the budget is spent; the warm-started trajectories that miss
  the target are solved again from the cold start inside the same run
  (`mmpc_batch_set_fallback`), and that second solve is charged.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import mlp, mmpc, scenes


@dataclass
class WarmConfig:
    train_scenes: int = 200_000
    goals_per_scene: int = 8
    obstacles: int = 50
    x_range: tuple = (-50.0, 250.0)
    steps: int = 4000
    batch: int = 4096
    lr: float = 1e-3
    lr_min: float = 1e-5
    weight_decay: float = 1e-4
    hidden: tuple = (256, 256, 256)
    predict_lam: bool = False     # False: the network predicts c; lambda^0 = Q c^0 (or 0, lam_from_q False)
    lam_from_q: bool = True
    converged_only: bool = True   # train on the trajectories that reached tol only
    tensor_inference: bool = True  # inference on the tensor cores (tcgen05, bfloat16 layer inputs)
    tensor_training: bool = True   # training products on the tensor cores (bfloat16 operands)
    tol: float = 1e-2
    seed: int = 0
    params: dict = field(default_factory=lambda: dict(scenes.BASE_PARAMS))

    @property
    def outputs(self) -> int:
        return (6 if self.predict_lam else 3) * int(self.params["n"])

    @property
    def widths(self) -> tuple:
        return (64,) + tuple(self.hidden) + (self.outputs,)


def _dev(a, device, dtype=None):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device=device).contiguous()


class WarmStart:
    """A trained network with its output standardisation, producing warm
    starts for stacked scenes."""

    def __init__(self, net: mlp.Mlp, mu, sigma, params: dict, Q=None):
        self.net, self.mu, self.sigma, self.params, self.Q = net, mu, sigma, dict(params), Q
        self.n = int(params["n"])
        self.outputs = int(mu.numel())

    def buffers(self, S: int, B: int, device):
        import torch
        n = self.n
        return dict(X=torch.zeros((S, B, 64), device=device), Y=torch.zeros((S, B, self.outputs), device=device),
                    coef=torch.zeros((S, B, 3 * n), device=device), lam=torch.zeros((S, B, 3 * n), device=device))

    def predict(self, ego, obst, goals, buf, table=None, stream=None):
        """Warm starts into buf["coef"], buf["lam"] (enqueue only; the
        returned descriptor table must outlive the launches)."""
        S, B = int(goals.shape[0]), int(goals.shape[1])
        if table is None:
            table = mlp.uniform_table(goals.device, ego=ego, obst=obst, goals=goals, X=buf["X"], Y=buf["Y"],
                                      coef=buf["coef"], lam=buf["lam"])
        mlp.features(table, self.params["a"], self.params["b"], stream)
        self.net.forward(buf["X"].view(S * B, 64), buf["Y"].view(S * B, self.outputs), stream)
        mlp.warm_decode(table, self.n, self.params["T"], self.mu, self.sigma, Q=self.Q, stream=stream)
        return table

    def close(self):
        self.net.close()


def q_matrix(params: dict, device):
    """Q = Pdd^T Pdd of the problem (mmpc_build), device float32 [n, n]."""
    import torch
    n, N = int(params["n"]), int(params["N"])
    buf = mmpc.mmpc_build(mmpc.make_params(**params), 0)
    o = N + 3 * N * n + n  # layout of mmpc_build: t, P, Pd, Pdd, lin, Q, ...
    return torch.tensor(buf[o:o + n * n].reshape(n, n).astype(np.float32), device=device).contiguous()


def build_dataset(cfg: WarmConfig, device, seed_offset: int = 0, S: int | None = None):
    """Feature rows X [R, 64] and raw encoded targets T [R, outputs]
    (R = S x goals, fewer with converged_only) from scenes solved by the
    plain method (100 iterations from the cold start)."""
    import torch
    S = cfg.train_scenes if S is None else S
    G = cfg.goals_per_scene
    n = int(cfg.params["n"])
    W = cfg.outputs
    p = dict(cfg.params)
    p.update(tol=0.0, check_every=10)
    X = torch.zeros((S, G, 64), device=device)
    T = torch.zeros((S, G, W), device=device)
    keep = torch.zeros((S, G), dtype=torch.bool, device=device)
    chunk = 16384
    meta = mmpc.make_meta(**scenes.META_ABS)
    zero, one = torch.zeros(W, device=device), torch.ones(W, device=device)
    for s0 in range(0, S, chunk):
        k = min(chunk, S - s0)
        ego, obst, goals = scenes.scene_stack(cfg.seed * 1_000_003 + seed_offset + s0, k, G, cfg.obstacles,
                                              cfg.x_range)
        ego, obst, goals = _dev(ego, device), _dev(obst, device), _dev(goals, device)
        bt = mmpc.Batch.from_uniform(p, ego, obst, goals, meta, want_lam=True)
        bt.run()
        coef = bt.flat["coef"].view(k, G, 3 * n)
        lam = bt.flat["lam"].view(k, G, 3 * n)
        tab = mlp.uniform_table(device, ego=ego, obst=obst, goals=goals, X=X[s0:s0 + k], coef=coef, lam=lam,
                                Z=T[s0:s0 + k])
        mlp.features(tab, p["a"], p["b"])
        mlp.warm_encode(tab, n, p["T"], zero, one)
        keep[s0:s0 + k] = (bt.flat["resid"][:, :3].max(dim=1).values <= cfg.tol).view(k, G)
        torch.cuda.synchronize(device)
        bt.close()
    X, T = X.view(S * G, 64), T.view(S * G, W)
    if cfg.converged_only:
        idx = torch.nonzero(keep.view(-1)).view(-1).to(torch.int32)
        Xk = torch.empty((idx.numel(), 64), device=device)
        Tk = torch.empty((idx.numel(), W), device=device)
        mlp.gather_rows(X, idx, Xk)
        mlp.gather_rows(T, idx, Tk)
        return Xk, Tk
    return X, T


def train(cfg: WarmConfig, X, T, device, log_every: int = 250):
    """Trains a network on (X, T); returns the WarmStart and the loss log."""
    import torch
    W = cfg.outputs
    R = int(X.shape[0])
    mu, sigma = torch.zeros(W, device=device), torch.ones(W, device=device)
    mlp.column_stats(T, mu, sigma)
    Z = torch.empty_like(T)
    mlp.standardize(T, mu, sigma, Z)
    Ws, bs = scenes.mlp_init(cfg.seed, cfg.widths)
    net = mlp.Mlp(cfg.widths, Ws, bs, max_batch=cfg.batch, weight_decay=cfg.weight_decay)
    net.set_train_tensor_cores(cfg.tensor_training)
    rng = np.random.default_rng(cfg.seed + 7)
    Xb = torch.zeros((cfg.batch, 64), device=device)
    Zb = torch.zeros((cfg.batch, W), device=device)
    loss = torch.zeros((1,), device=device)
    perm, pos = None, R
    log = []
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record()
    for step in range(cfg.steps):
        if pos + cfg.batch > R:
            perm = torch.tensor(rng.permutation(R).astype(np.int32), device=device)
            pos = 0
        idx = perm[pos:pos + cfg.batch]
        pos += cfg.batch
        mlp.gather_rows(X, idx, Xb)
        mlp.gather_rows(Z, idx, Zb)
        net.loss_grad(Xb, Zb, loss)
        lr = cfg.lr_min + 0.5 * (cfg.lr - cfg.lr_min) * (1 + math.cos(math.pi * step / max(1, cfg.steps)))
        net.adamw(lr)
        if step % log_every == 0 or step == cfg.steps - 1:
            log.append((step, float(loss.item())))
    t_end.record()
    torch.cuda.synchronize(device)
    Q = q_matrix(cfg.params, device) if (not cfg.predict_lam and cfg.lam_from_q) else None
    net.set_tensor_cores(cfg.tensor_inference)
    ws = WarmStart(net, mu, sigma, cfg.params, Q)
    # device time per training step (row gathers, loss and gradients, AdamW)
    ws.train_step_ms = t_start.elapsed_time(t_end) / max(1, cfg.steps)
    return ws, log


def time_forward(ws: WarmStart, rows: int, device, reps: int = 5):
    """Milliseconds of one network forward over `rows` feature rows, on the
    SIMT path and on the tensor cores (median of reps, CUDA events)."""
    import torch
    X = torch.randn((rows, 64), device=device)
    Y = torch.empty((rows, ws.outputs), device=device)
    out = {}
    for tag, on in (("simt_ms", False), ("tensor_ms", True)):
        ws.net.set_tensor_cores(on)
        ws.net.forward(X, Y)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ws.net.forward(X, Y)
            b.record()
            torch.cuda.synchronize(device)
            ts.append(a.elapsed_time(b))
        out[tag] = float(np.median(ts))
    ws.net.status()
    out["rows"] = rows
    out["flops"] = 2.0 * rows * sum(i * o for i, o in zip(ws.net.widths[:-1], ws.net.widths[1:]))
    ws.net.set_tensor_cores(True)
    return out


def validation_loss(ws: WarmStart, X, T):
    """Mean squared error of the network's standardised outputs on (X, T),
    by the network's own loss kernel in chunks of its batch size."""
    import torch
    Z = torch.empty_like(T)
    mlp.standardize(T, ws.mu, ws.sigma, Z)
    loss = torch.zeros((1,), device=X.device)
    R, mb, acc = int(X.shape[0]), ws.net.max_batch, 0.0
    for r0 in range(0, R, mb):
        k = min(mb, R - r0)
        ws.net.loss_grad(X[r0:r0 + k], Z[r0:r0 + k], loss)
        acc += float(loss.item()) * k
    return acc / R


def evaluate(ws: WarmStart, cfg: WarmConfig, device, S: int = 4096, B: int = 256, seed: int = 10**6,
             reps: int = 3, tol: float = 1e-2, obstacles=None, x_range=None, plain: bool = False,
             stall: tuple | None = None, keep: bool = False, precision: int = 0, near: float = 5.0):
    """Cold start against warm start (+ cold fallback) on S fresh scenes x B
    goals, each timed as one CUDA graph replay (warm: features, network,
    decode, solve, fallback solve, score).  Returns a dict of results.  With
    the stall stop, a fourth variant falls back only the misses that ran the
    whole budget (`warm_fallback_budget`, mmpc_batch_set_fallback mode 2), and a
    fifth only the near misses among those, residual <= near x tol
    (`warm_fallback_near`, mode 3).
    With precision (an MMPC_PREC_* other than FP32), the batched solves run on
    the tensor-core kernel (variant 3); the plain method and the cold fallback
    stay FP32.  With keep, out["_keep"] holds the warm-started batch, its step function,
    the graphs per variant and the inputs, for the caller to time further and
    close."""
    import torch
    m = cfg.obstacles if obstacles is None else obstacles
    xr = cfg.x_range if x_range is None else x_range
    ego, obst, goals = scenes.scene_stack(seed, S, B, m, xr, goals="grid" if B % 8 == 0 else "random")
    ego, obst, goals = _dev(ego, device), _dev(obst, device), _dev(goals, device)
    p = dict(cfg.params)
    p.update(tol=tol, check_every=10)
    pb = dict(p)  # the batched variants: with the opt-in stall stop when given
    if stall is not None:
        pb.update(stall_tol=float(stall[0]), stall_ratio=float(stall[1]))
    if precision:  # the batched solves on the tensor cores (variant 3) in that precision
        pb.update(variant=3, precision=int(precision))
    meta = mmpc.make_meta(**scenes.META_ABS)
    stream = torch.cuda.Stream(device)
    out = {}

    def timed(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            fn()  # warm-up outside the graph
        torch.cuda.synchronize(device)
        with torch.cuda.graph(g, stream=stream):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        times = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                g.replay()
                ev[1].record(stream)
            torch.cuda.synchronize(device)
            times.append(ev[0].elapsed_time(ev[1]))
        return g, float(np.median(times))

    def stats(bt, ms, tag):
        resid = bt.flat["resid"].view(-1, 4)
        conv = (resid[:, :3].max(dim=1).values <= tol)
        it = bt.flat["iters"].to(torch.int64)
        out[tag] = dict(ms=ms, trajectories=S * B, trajectories_per_s=S * B / (ms * 1e-3),
                        converged=int(conv.sum().item()), converged_per_s=int(conv.sum().item()) / (ms * 1e-3),
                        mean_iters=float(it.double().mean().item()),
                        mean_iters_converged=float(it[conv].double().mean().item()) if conv.any() else None)

    if plain:
        # the plain method: one mmpc_solve + mmpc_score per scene, back to back
        # on one stream (captured in a graph, so host launch cost is not counted)
        n = int(p["n"])
        sv = mmpc.Solver(p, m)
        pc = torch.zeros((S, B, 3 * n), device=device)
        pr = torch.zeros((S, B, 4), device=device)
        pi = torch.zeros((S, B), dtype=torch.int32, device=device)
        pcost = torch.zeros((S, B), device=device)
        pam = torch.zeros((S, 1), dtype=torch.int32, device=device)

        def plain_step():
            for i in range(S):
                mmpc.mmpc_solve(sv.ctx, ego[i], obst[i] if m else None, goals[i], pc[i], None, None, None, pr[i],
                                pi[i])
                mmpc.mmpc_score(sv.ctx, meta, pc[i], pcost[i], pam[i])
        g_plain, ms = timed(plain_step)
        conv = (pr.view(-1, 4)[:, :3].max(dim=1).values <= tol)
        out["plain"] = dict(ms=ms, trajectories=S * B, trajectories_per_s=S * B / (ms * 1e-3),
                            converged=int(conv.sum().item()), converged_per_s=int(conv.sum().item()) / (ms * 1e-3),
                            launches=2 * S)
        del g_plain
        sv.close()

    cold = mmpc.Batch.from_uniform(pb, ego, obst, goals, meta)
    g_cold, ms = timed(cold.run)
    stats(cold, ms, "cold")
    cold_conv = (cold.flat["resid"].view(-1, 4)[:, :3].max(dim=1).values <= tol)

    buf = ws.buffers(S, B, device)
    warm = mmpc.Batch.from_uniform(pb, ego, obst, goals, meta, warm_coef=buf["coef"], warm_lam=buf["lam"])
    table = mlp.uniform_table(device, ego=ego, obst=obst, goals=goals, X=buf["X"], Y=buf["Y"], coef=buf["coef"],
                              lam=buf["lam"])

    def warm_step():
        ws.predict(ego, obst, goals, buf, table=table)
        warm.run()

    warm.set_fallback(False)
    g_w, ms = timed(warm_step)
    stats(warm, ms, "warm")
    warm_resid = warm.flat["resid"].view(-1, 4)[:, :3].max(dim=1).values.clone()
    warm_conv = warm_resid <= tol
    warm_iters = warm.flat["iters"].clone()
    out["warm"]["misses"] = int((~warm_conv).sum().item())
    del g_w
    g_fb2 = None
    if stall is not None:
        # only the misses that ran the whole budget go to the cold fallback
        warm.set_fallback(2)
        g_fb2, ms = timed(warm_step)
        stats(warm, ms, "warm_fallback_budget")
        out["warm_fallback_budget"]["fallbacks"] = warm.fallbacks()
        budget_miss = (~warm_conv) & (warm_iters == int(pb["iters"]))
        out["warm_fallback_budget"]["budget_misses"] = int(budget_miss.sum().item())
        out["warm_fallback_budget"]["passes"] = int((warm_iters.to(torch.int64) + 1).sum().item() +
                                                    (cold.flat["iters"].to(torch.int64) + 1)[budget_miss].sum().item())
    g_fb3 = None
    if stall is not None:
        # only the near misses (residual <= near x tol) that ran the whole budget
        warm.set_fallback(3, near=near)
        g_fb3, ms = timed(warm_step)
        stats(warm, ms, "warm_fallback_near")
        out["warm_fallback_near"]["fallbacks"] = warm.fallbacks()
        out["warm_fallback_near"]["near"] = near
        near_miss = (~warm_conv) & (warm_iters == int(pb["iters"])) & (warm_resid <= near * tol)
        out["warm_fallback_near"]["passes"] = int((warm_iters.to(torch.int64) + 1).sum().item() +
                                                  (cold.flat["iters"].to(torch.int64) + 1)[near_miss].sum().item())
    warm.set_fallback(True)
    g_f, ms = timed(warm_step)
    stats(warm, ms, "warm_fallback")
    out["warm_fallback"]["fallbacks"] = warm.fallbacks()
    # the fallback re-solves exactly the misses, from the cold start
    fb_match = bool(torch.equal(warm.flat["coef"].view(S * B, -1)[~warm_conv],
                                cold.flat["coef"].view(S * B, -1)[~warm_conv]))
    out["warm_fallback"]["fallback_equals_cold"] = fb_match
    # AM passes (initial + one per iteration) each run spent, for the roofline
    cold_passes = cold.flat["iters"].to(torch.int64) + 1
    warm_passes = warm_iters.to(torch.int64) + 1
    out["cold"]["passes"] = int(cold_passes.sum().item())
    out["warm"]["passes"] = int(warm_passes.sum().item())
    out["warm_fallback"]["passes"] = int(warm_passes.sum().item() + cold_passes[~warm_conv].sum().item())
    both = cold_conv & warm_conv
    out["converged_both"] = int(both.sum().item())
    out["converged_warm_only"] = int((warm_conv & ~cold_conv).sum().item())
    out["converged_cold_only"] = int((cold_conv & ~warm_conv).sum().item())
    if both.any():
        out["iters_both_converged"] = dict(cold=float(cold.flat["iters"][both].double().mean().item()),
                                           warm=float(warm_iters[both].double().mean().item()))
    out["scenes"], out["goals"], out["obstacles"], out["x_range"] = S, B, m, list(xr)
    out["stall"] = None if stall is None else list(stall)
    out["precision"] = int(precision)
    out["speedup_trajectories_per_s"] = out["warm_fallback"]["trajectories_per_s"] / out["cold"]["trajectories_per_s"]
    if plain:
        out["batched_cold_vs_plain"] = out["cold"]["trajectories_per_s"] / out["plain"]["trajectories_per_s"]
        out["batched_warm_fallback_vs_plain"] = (out["warm_fallback"]["trajectories_per_s"] /
                                                 out["plain"]["trajectories_per_s"])
        out["batched_warm_vs_plain"] = out["warm"]["trajectories_per_s"] / out["plain"]["trajectories_per_s"]
    if out["cold"]["converged"] > 0:
        out["speedup_converged_per_s"] = out["warm_fallback"]["converged_per_s"] / out["cold"]["converged_per_s"]
    if keep:
        out["_keep"] = dict(warm=warm, cold=cold, step=warm_step, stream=stream, table=table, buf=buf,
                            graphs=dict(cold=g_cold, warm_fallback=g_f, warm_fallback_budget=g_fb2,
                                        warm_fallback_near=g_fb3),
                            inputs=dict(ego=ego, obst=obst, goals=goals))
        return out
    del g_cold, g_f, g_fb2, g_fb3
    cold.close()
    warm.close()
    return out


def run(cfg: WarmConfig, device, eval_kwargs: list | None = None, log=print):
    """Dataset, training, validation and evaluation; returns a report."""
    t0 = time.perf_counter()
    X, T = build_dataset(cfg, device)
    t1 = time.perf_counter()
    ws, losses = train(cfg, X, T, device)
    import torch
    torch.cuda.synchronize(device)
    t2 = time.perf_counter()
    Xv, Tv = build_dataset(cfg, device, seed_offset=7_777_777, S=max(256, cfg.train_scenes // 50))
    report = dict(dataset_s=t1 - t0, train_s=t2 - t1, rows=int(X.shape[0]), losses=losses,
                  val_loss=validation_loss(ws, Xv, Tv), evals=[])
    for kw in eval_kwargs or [{}]:
        report["evals"].append(evaluate(ws, cfg, device, **kw))
    ws.close()
    return report
