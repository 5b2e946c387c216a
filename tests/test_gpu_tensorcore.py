"""The tensor-core solve kernel (variant 3): the shared-matrix products of
Algorithm 1 (the evaluations P c and the contractions P^T e of Eqs.
lin_solve_xy_2 / lin_solve_psi_2) as tcgen05.mma in TF32 or BF16 with FP32
accumulation, optionally as hi + lo splits; projections, QP steps and
multipliers FP32.  Checked against the FP64 oracle:

* ragged shapes (N not a multiple of the 16-sample chunk, n < 12 and n = 16,
  no obstacles, B smaller than a tile): TF32 hi + lo to the FP32 parity bars,
  BF16 hi + lo (16 significant bits per product) to 1e-2 m;
* the precision workload (16384 goals, 30 obstacles, N = 200, n = 16) at its
  full size, every 256th trajectory: the error table of the four modes, with
  TF32 hi + lo (and the FP32 kernel) within 1e-3 m on the whole parity set,
  BF16 hi + lo on 95 % of it, and the unsplit BF16 mode missing the bar;
* a trajectory's result does not depend on its slot in the tile (the goals
  are bucket-sorted into warps; permuting the goals permutes the results bit
  for bit);
* arguments the kernel cannot take are refused at setup.
"""
import numpy as np
import pytest

import parity_utils as U
from paper_2109_10392_gb300 import mmpc, scenes

pytestmark = pytest.mark.gpu

NAMES = {mmpc.MMPC_PREC_TF32: "tf32", mmpc.MMPC_PREC_TF32_SPLIT: "tf32 hi+lo", mmpc.MMPC_PREC_BF16: "bf16",
         mmpc.MMPC_PREC_BF16_SPLIT: "bf16 hi+lo"}

BF16_TOL = 1e-2  # [m] positions of the BF16 hi + lo mode on the parity set

# (N, n, m, B, iters): ragged chunk tails, both coefficient paddings, no obstacles
SHAPES = [
    (16, 7, 0, 3, 30),
    (37, 10, 3, 5, 25),
    (100, 12, 4, 40, 40),
    (130, 12, 5, 3, 20),
    (200, 16, 8, 4, 20),
    (64, 13, 2, 3, 15),
]


@pytest.mark.parametrize("prec", [mmpc.MMPC_PREC_TF32_SPLIT, mmpc.MMPC_PREC_BF16_SPLIT])
@pytest.mark.parametrize("N,n,m,B,iters", SHAPES)
def test_shapes_split_modes(N, n, m, B, iters, prec):
    sc = scenes.scene_custom(seed=N + n + m, B=B, m=m, N=N, n=n, x_range=(10.0, 150.0))
    params = dict(sc.params, iters=iters)
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)
    orc = U.oracle_solve(params, ego, obst, goals)
    gpu = U.gpu_solve(dict(params, variant=3, precision=prec), ego, obst, goals)
    assert np.array_equal(gpu["iters"], orc["iters"])
    if prec == mmpc.MMPC_PREC_TF32_SPLIT:
        # 22 significant bits per product: the FP32 parity bars
        U.check_parity(params, ego, obst, goals, gpu, orc)
    else:
        # BF16 hi + lo carries 16 significant bits: a 100 m position term
        # keeps about 1e-3 m, so the bar is BF16_TOL on the parity set
        err = U.pos_err(params, gpu["coef"], orc["coef"])
        sens = U.sensitivity(params, ego, obst, goals, orc["coef"])
        good = sens < U.SENS_TOL
        assert good.mean() >= 0.3
        assert np.all(err[good] <= BF16_TOL), err
        assert np.all(np.isfinite(gpu["coef"]))
        assert np.all(U.boundary_error(params, ego, goals, gpu["coef"]) < 1e-2)


def test_eleven_goal_scene_tf32_split():
    sc = scenes.scene_small(0)
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)
    params = dict(sc.params, tol=0.0)
    orc = U.oracle_solve(params, ego, obst, goals)
    gpu = U.gpu_solve(dict(params, variant=3, precision=mmpc.MMPC_PREC_TF32_SPLIT), ego, obst, goals)
    U.check_parity(params, ego, obst, goals, gpu, orc)
    rel = np.abs(gpu["resid"] - orc["resid"]) / np.maximum(np.abs(orc["resid"]), 1e-3)
    assert np.median(rel) < 1e-2


def test_precision_workload_error_table(capsys):
    sc = scenes.scene_custom(31, 16384, 30, N=200, n=16)
    params = dict(sc.params, tol=0.0)
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)
    sel = np.arange(0, len(goals), 256)
    orc = U.oracle_solve(params, ego, obst, goals[sel])
    sens = U.sensitivity(params, ego, obst, goals[sel], orc["coef"], trials=1)
    good = sens < U.SENS_TOL
    fp32 = U.gpu_solve(params, ego, obst, goals)
    err32 = U.pos_err(params, fp32["coef"][sel], orc["coef"])
    rows = [f"  {'fp32 (CUDA cores)':>18}: parity set ({good.sum()}) median {np.median(err32[good]):.2e} max "
            f"{err32[good].max():.2e} m, share <= 1e-3 m {np.mean(err32[good] <= U.POS_TOL):.2f}"]
    med, share = {}, {}
    for mode in NAMES:
        gpu = U.gpu_solve(dict(params, variant=3, precision=mode), ego, obst, goals)
        assert np.all(np.isfinite(gpu["coef"])), NAMES[mode]
        err = U.pos_err(params, gpu["coef"][sel], orc["coef"])
        med[mode] = float(np.median(err[good]))
        share[mode] = float(np.mean(err[good] <= U.POS_TOL))
        rows.append(f"  {NAMES[mode] + ' (tensor)':>18}: parity set ({good.sum()}) median {med[mode]:.2e} max "
                    f"{err[good].max():.2e} m, share <= 1e-3 m {share[mode]:.2f}; all sampled median "
                    f"{np.median(err):.2e} m")
    with capsys.disabled():
        print(f"\n[tensor-core modes, N = 200, n = 16, m = 30, sample {len(sel)} of 16384]")
        print("\n".join(rows))
    tf32, tf32s, bf16, bf16s = (mmpc.MMPC_PREC_TF32, mmpc.MMPC_PREC_TF32_SPLIT, mmpc.MMPC_PREC_BF16,
                                mmpc.MMPC_PREC_BF16_SPLIT)
    m32 = float(np.median(err32[good]))
    # the splits keep FP32-class positions (TF32 hi + lo and the FP32 kernel
    # on the FP32 bar over the whole parity set); the plain types do not
    assert np.all(err32[good] <= U.POS_TOL), err32[good]
    assert share[tf32s] == 1.0 and share[bf16s] >= 0.95
    assert med[tf32s] <= 2 * m32 and med[bf16s] <= 2 * m32
    assert med[tf32s] <= med[tf32] and med[bf16s] <= med[bf16]
    assert share[bf16] < 0.5 and med[bf16] > 1e-3


def test_result_independent_of_slot():
    """Permuting the goals permutes the results bit for bit (slot order,
    tile and warp membership do not enter a trajectory's arithmetic)."""
    sc = scenes.scene_custom(7, 700, 12, N=100, n=12)
    params = dict(sc.params, tol=1e-2, variant=3, precision=mmpc.MMPC_PREC_BF16_SPLIT)
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)
    a = U.gpu_solve(params, ego, obst, goals)
    perm = np.random.default_rng(3).permutation(len(goals))
    b = U.gpu_solve(params, ego, obst, goals[perm])
    for k in ("coef", "lam", "resid", "iters"):
        assert np.array_equal(a[k][perm], b[k]), k


def test_early_exit_matches_oracle_iterations():
    sc = scenes.scene_custom(11, 48, 3, N=100, n=12, x_range=(30.0, 200.0))
    params = dict(sc.params, tol=1e-2, check_every=10)
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)
    gpu = U.gpu_solve(dict(params, variant=3, precision=mmpc.MMPC_PREC_TF32_SPLIT), ego, obst, goals)
    orc = U.oracle_solve(params, ego, obst, goals)
    conv = orc["iters"] < params["iters"]
    assert conv.sum() >= 10
    # converging trajectories stop at the same check as the oracle (or the next)
    assert np.all(np.abs(gpu["iters"][conv] - orc["iters"][conv]) <= params["check_every"])


def test_arguments():
    base = dict(scenes.scene_custom(1, 4, 3, N=100, n=12).params)
    for bad in (dict(base, variant=3, precision=0), dict(base, variant=3, precision=2, N=300),
                dict(base, variant=4, precision=2)):
        with pytest.raises(mmpc.MmpcError):
            mmpc.Solver(bad, 3)
    with pytest.raises(mmpc.MmpcError):
        mmpc.Solver(dict(base, variant=3, precision=2), 129)
    s = mmpc.Solver(dict(base, variant=3, precision=4), 128)
    s.close()


def _batch(params, ego, obst, goals, warm_coef=None, warm_lam=None):
    import torch
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda:0").contiguous()  # noqa: E731
    return mmpc.Batch.from_uniform(params, t(ego), t(obst), t(goals), scenes.META_ABS, want_lam=True,
                                   warm_coef=warm_coef, warm_lam=warm_lam)


def test_batch_matches_single_scene_solves():
    """A batch of scenes on the tensor-core kernel (one persistent launch over
    all scenes' 32-goal items, uneven last items) reproduces each scene
    solved alone, bit for bit, and the same again when replayed from a CUDA
    graph."""
    import torch
    S, B, m = 6, 70, 8
    ego, obst, goals = scenes.scene_stack(5, S, B, m, (10.0, 150.0))
    ego, obst, goals = U.f32(ego), U.f32(obst), U.f32(goals)
    params = dict(scenes.BASE_PARAMS, tol=1e-2, variant=3, precision=mmpc.MMPC_PREC_TF32_SPLIT)
    bt = _batch(params, ego, obst, goals)
    bt.run()
    torch.cuda.synchronize()
    first = {k: bt.flat[k].clone() for k in ("coef", "lam", "resid", "iters", "cost")}
    n = params["n"]
    for s in range(S):
        one = U.gpu_solve(params, ego[s], obst[s], goals[s])
        sl = slice(s * B, (s + 1) * B)
        assert np.array_equal(first["coef"].view(-1, 3 * n)[sl].double().cpu().numpy(), one["coef"])
        assert np.array_equal(first["lam"].view(-1, 3 * n)[sl].double().cpu().numpy(), one["lam"])
        assert np.array_equal(first["resid"].view(-1, 4)[sl].double().cpu().numpy(), one["resid"])
        assert np.array_equal(first["iters"][sl].cpu().numpy(), one["iters"])
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        bt.run()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=st):
        bt.run()
    g.replay()
    torch.cuda.synchronize()
    for k, v in first.items():
        assert torch.equal(bt.flat[k], v), k
    bt.status()
    bt.close()


def test_batch_against_oracle_with_warm_start_and_fallback():
    """Warm-started tensor-core batch with the FP32 cold fallback of the
    misses: converged trajectories and the re-solved misses both match the
    oracle (positions on the parity set)."""
    import torch
    S, B, m = 3, 40, 6
    ego, obst, goals = scenes.scene_stack(9, S, B, m, (10.0, 150.0))
    ego, obst, goals = U.f32(ego), U.f32(obst), U.f32(goals)
    params = dict(scenes.BASE_PARAMS, tol=1e-2, variant=3, precision=mmpc.MMPC_PREC_TF32_SPLIT)
    # warm starts: the oracle's own solutions at 10 iterations (a start off the
    # boundary rows' exact values is projected by the first step)
    p10 = dict(params, iters=10, tol=0.0)
    n = params["n"]
    wc = np.zeros((S, B, 3 * n)); wl = np.zeros((S, B, 3 * n))
    for s in range(S):
        r = U.oracle_solve(p10, ego[s], obst[s], goals[s])
        wc[s], wl[s] = r["coef"], r["lam"]
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda:0").contiguous()  # noqa: E731
    bt = _batch(params, ego, obst, goals, warm_coef=t(wc), warm_lam=t(wl))
    bt.set_fallback(True)
    bt.run()
    torch.cuda.synchronize()
    coef = bt.flat["coef"].view(S, B, 3 * n).double().cpu().numpy()
    for s in range(S):
        orc_w = U.oracle_solve(params, ego[s], obst[s], goals[s], init=U.f32(wc[s]), init_lam=U.f32(wl[s]))
        orc_c = U.oracle_solve(params, ego[s], obst[s], goals[s])
        conv = orc_w["resid"][:, :3].max(axis=1) <= params["tol"]
        ref = np.where(conv[:, None], orc_w["coef"], orc_c["coef"])  # misses were solved again cold
        err = U.pos_err(params, coef[s], ref)
        sens = U.sensitivity(params, ego[s], obst[s], goals[s], orc_c["coef"], trials=1)
        good = (sens < U.SENS_TOL) & conv
        assert np.all(err[good] <= U.POS_TOL), err[good]
    bt.close()


def test_batch_schedules_and_autotune():
    """A batch of one variant-3 context runs on the tensor cores (schedule 5)
    or on the FP32 kernel (1-4, the same results as a context of variant 0);
    the autotuner times all five, and a second batch of the same signature
    takes the cached choice."""
    import torch
    S, B, m = 4, 64, 6
    ego, obst, goals = scenes.scene_stack(21, S, B, m, (10.0, 150.0))
    ego, obst, goals = U.f32(ego), U.f32(obst), U.f32(goals)
    p3 = dict(scenes.BASE_PARAMS, tol=1e-2, variant=3, precision=mmpc.MMPC_PREC_TF32_SPLIT)
    p0 = dict(scenes.BASE_PARAMS, tol=1e-2)
    ref = _batch(p0, ego, obst, goals)
    ref.run()
    bt = _batch(p3, ego, obst, goals)
    for sch in (1, 4):
        bt.set_schedule(sch)
        bt.run()
        torch.cuda.synchronize()
        for k in ("coef", "resid", "iters", "cost", "argmin"):
            assert torch.equal(bt.flat[k], ref.flat[k]), (sch, k)
    bt.set_schedule(5)
    bt.run()
    torch.cuda.synchronize()
    n = p3["n"]
    one = U.gpu_solve(p3, ego[0], obst[0], goals[0])
    assert np.array_equal(bt.flat["coef"].view(-1, 3 * n)[:B].double().cpu().numpy(), one["coef"])
    with pytest.raises(mmpc.MmpcError):
        ref.set_schedule(5)
    bt.set_schedule(5)
    d = bt.describe()
    assert d["schedule"] == 5 and len(d["launches"]) == 1
    x = d["launches"][0]
    assert x["kernel"] == "tensor cores" and x["threads"] == 384 and x["trajectories"] == S * B and x["grid"] >= 1
    chosen = bt.autotune()
    assert chosen in (1, 2, 3, 4, 5)
    again = _batch(p3, ego, obst, goals)
    assert again.autotune() == chosen
    for b_ in (ref, bt, again):
        b_.close()
