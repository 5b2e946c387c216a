"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs (rounded to float32 for both).

Bars, from the parity target of this path: positions within 1e-3 m after the
fixed iteration count, meta costs within 1e-4 relative, the same argmin --
on the trajectories whose result is determined by the inputs to better than
the FP32 rounding (parity set, see parity_utils); the others are checked for
validity.
"""
import numpy as np
import pytest

import oracle
import parity_utils as U
from paper_2109_10392_gb300 import scenes

pytestmark = pytest.mark.gpu


def _scene_arrays(sc):
    return U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)


_check_parity = U.check_parity


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_highway_11_goals_10_obstacles(seed, variant):
    sc = scenes.scene_small(seed)
    sc.params["variant"] = variant
    ego, obst, goals = _scene_arrays(sc)
    orc = U.oracle_solve(sc.params, ego, obst, goals)
    gpu = U.gpu_solve(sc.params, ego, obst, goals)
    err, good = _check_parity(sc.params, ego, obst, goals, gpu, orc)
    # residual outputs follow the oracle's definitions
    assert np.allclose(gpu["resid"][good], orc["resid"][good], rtol=1e-2, atol=2e-3)
    assert np.all(gpu["iters"] == sc.params["iters"])
    # meta cost and argmin
    cg, ag = U.gpu_score(sc.params, obst.shape[0], gpu["coef"], sc.meta)
    co, ao = U.meta_oracle(sc.params, orc["coef"], sc.meta)
    fin = np.isfinite(co) & good
    assert np.all(np.abs(cg[fin] - co[fin]) <= U.COST_RTOL * np.abs(co[fin]) + 1e-3)
    if ao >= 0 and good[ao]:
        second = np.sort(co[np.isfinite(co)])[1] if np.isfinite(co).sum() > 1 else np.inf
        if second - co[ao] > 2 * U.COST_RTOL * co[ao] + 2e-3:
            assert ag == ao
        else:
            assert abs(co[ag] - co[ao]) <= 2 * U.COST_RTOL * co[ao] + 2e-3


# (N, n, m, B, iters): several warps of samples with ragged tails, both
# coefficient paddings (12, 16), and every launch-bound variant (<=128, <=256,
# <=512 threads).
SHAPES = [
    (16, 7, 0, 3, 30),
    (37, 10, 3, 5, 25),
    (100, 12, 1, 4, 40),
    (130, 12, 5, 3, 20),
    (200, 16, 8, 4, 20),
    (64, 13, 2, 3, 15),
    (300, 12, 4, 2, 10),
    (512, 16, 2, 2, 6),
]


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("N,n,m,B,iters", SHAPES)
def test_shapes(N, n, m, B, iters, variant):
    if variant == 1 and N > 256:
        pytest.skip("the one-sample kernel covers N <= 256")
    sc = scenes.scene_custom(seed=N + n + m, B=B, m=m, N=N, n=n, x_range=(10.0, 150.0))
    params = dict(sc.params)
    params["iters"] = iters
    params["variant"] = variant
    ego, obst, goals = _scene_arrays(sc)
    orc = U.oracle_solve(params, ego, obst, goals)
    gpu = U.gpu_solve(params, ego, obst, goals)
    _check_parity(params, ego, obst, goals, gpu, orc)


@pytest.mark.parametrize("variant", [0, 2])
def test_full_size_sampled(variant, capsys):
    """The 1024-goal, 50-obstacle scene in the launch configuration the
    benchmark times (variant 0: automatic, as the benchmark runs it).  The
    oracle solves all 1024 goals: meta costs within 1e-4 relative on the
    parity set and the batch argmin over all goals, unconditionally (the GPU's
    choice is the oracle's, or the two costs are within the cost tolerance of
    each other); positions with the conditioning probe on every 8th goal,
    whose parity-set share is printed and held to 0.45 (measured 0.484)."""
    sc = scenes.scene_large(0)
    sc.params["variant"] = variant
    ego, obst, goals = _scene_arrays(sc)
    gpu = U.gpu_solve(sc.params, ego, obst, goals)
    orc_all = U.oracle_solve(sc.params, ego, obst, goals)
    sel = np.arange(0, len(goals), 8)
    orc = {k: v[sel] for k, v in orc_all.items()}
    sens = U.sensitivity(sc.params, ego, obst, goals[sel], orc["coef"])
    gs = {k: v[sel] for k, v in gpu.items()}
    err, good = _check_parity(sc.params, ego, obst, goals[sel], gs, orc, sens=sens, min_frac=0.45)
    cg, ag = U.gpu_score(sc.params, obst.shape[0], gpu["coef"], sc.meta)
    co, ao = U.meta_oracle(sc.params, orc_all["coef"], sc.meta)
    fin = np.isfinite(co[sel]) & good
    rel = np.abs(cg[sel][fin] - co[sel][fin]) / np.maximum(np.abs(co[sel][fin]), 1e-9)
    with capsys.disabled():
        print(f"\n[1024 goals, variant {variant}] parity set {good.mean():.3f} of {len(sel)}; position error "
              f"max {err[good].max():.2e} m; meta cost rel error max {rel.max():.2e}; argmin gpu {ag} "
              f"oracle {ao} (costs {co[ag]:.6g} / {co[ao]:.6g})")
    assert np.all(rel <= U.COST_RTOL)
    assert ao >= 0 and ag >= 0
    assert ag == ao or abs(co[ag] - co[ao]) <= U.COST_RTOL * abs(co[ao])


def test_cold_start_only():
    sc = scenes.scene_small(5)
    params = dict(sc.params)
    params["iters"] = 0
    ego, obst, goals = _scene_arrays(sc)
    orc = U.oracle_solve(params, ego, obst, goals)
    gpu = U.gpu_solve(params, ego, obst, goals)
    assert np.all(U.pos_err(params, gpu["coef"], orc["coef"]) < 1e-4)
    assert np.allclose(gpu["resid"], orc["resid"], rtol=1e-3, atol=1e-3)
    assert np.all(gpu["iters"] == 0)
    assert np.allclose(gpu["lam"], 0.0)


def test_warm_start_continues_the_iteration():
    sc = scenes.scene_small(6)
    ego, obst, goals = _scene_arrays(sc)
    p10 = dict(sc.params); p10["iters"] = 10
    p5 = dict(sc.params); p5["iters"] = 5
    r10 = U.oracle_solve(p10, ego, obst, goals)
    c10, l10 = U.f32(r10["coef"]), U.f32(r10["lam"])
    orc = U.oracle_solve(p5, ego, obst, goals, init=c10, init_lam=l10)
    gpu = U.gpu_solve(p5, ego, obst, goals, warm_coef=c10, warm_lam=l10)
    _check_parity(p5, ego, obst, goals, gpu, orc, init=c10, init_lam=l10)


def test_warm_start_off_the_boundary_rows():
    """A warm start that violates A c = b is put back on the boundary rows by
    the first step, as Eq. lin_solve_xy_2 does from any iterate."""
    sc = scenes.scene_small(7)
    ego, obst, goals = _scene_arrays(sc)
    params = dict(sc.params); params["iters"] = 8
    rng = np.random.default_rng(0)
    warm = U.f32(U.oracle_solve(dict(params, iters=0), ego, obst, goals)["coef"] + rng.normal(scale=0.5, size=(len(goals), 36)))
    orc = U.oracle_solve(params, ego, obst, goals, init=warm)
    gpu = U.gpu_solve(params, ego, obst, goals, warm_coef=warm)
    _check_parity(params, ego, obst, goals, gpu, orc, init=warm)
    assert np.all(U.boundary_error(params, ego, goals, gpu["coef"]) < 1e-3)


def test_early_exit_matches_fixed_count():
    sc = scenes.scene_small(8)
    params = dict(sc.params); params.update(tol=1e-2, check_every=5)
    ego, obst, goals = _scene_arrays(sc)
    gpu = U.gpu_solve(params, ego, obst, goals)
    it = gpu["iters"]
    assert np.all((it % 5 == 0) | (it == params["iters"]))
    conv = np.max(gpu["resid"][:, :3], axis=1)
    early = it < params["iters"]
    assert np.all(conv[early] <= 1e-2)
    for K in np.unique(it):
        idx = np.where(it == K)[0]
        pk = dict(sc.params); pk["iters"] = int(K)
        orc = U.oracle_solve(pk, ego, obst, goals[idx])
        err = U.pos_err(pk, gpu["coef"][idx], orc["coef"])
        assert np.all(err <= U.POS_TOL), (K, err.max())


def test_colocated_obstacle_degenerate_projection():
    """Ego and an obstacle at the same place with the same velocity: every
    sample has w = 0, where alpha = atan2(0, 0) = 0 and d = 1, so each sample
    contributes a to the obstacle residual: r_obs = a sqrt(N) at the start."""
    params = dict(scenes.BASE_PARAMS); params["iters"] = 0
    ego = np.array([0.0, 15.0, 0.0, 0.0])
    obst = np.array([[0.0, 0.0, 15.0, 0.0]])
    goals = np.array([[0.0, 15.0, 0.0]])
    gpu = U.gpu_solve(params, ego, obst, goals)
    orc = U.oracle_solve(params, ego, obst, goals)
    expect = params["a"] * np.sqrt(params["N"])
    assert np.isclose(gpu["resid"][0, 0], expect, rtol=1e-5)
    assert np.isclose(orc["resid"][0, 0], expect, rtol=1e-9)
    params["iters"] = 20
    gpu = U.gpu_solve(params, ego, obst, goals)
    assert np.all(np.isfinite(gpu["coef"])) and np.all(np.isfinite(gpu["resid"]))
    assert np.all(U.boundary_error(params, ego, goals, gpu["coef"]) < 1e-3)


def test_batch_independence_and_determinism():
    sc = scenes.scene_small(9)
    ego, obst, goals = _scene_arrays(sc)
    a = U.gpu_solve(sc.params, ego, obst, goals)
    b = U.gpu_solve(sc.params, ego, obst, goals)
    assert np.array_equal(a["coef"], b["coef"])
    perm = np.random.default_rng(3).permutation(len(goals))
    c = U.gpu_solve(sc.params, ego, obst, goals[perm])
    assert np.array_equal(a["coef"][perm], c["coef"])
    d = U.gpu_solve(sc.params, ego, obst, goals[:3])
    assert np.array_equal(a["coef"][:3], d["coef"])


def test_nan_goal_never_wins():
    sc = scenes.scene_small(10)
    ego, obst, goals = _scene_arrays(sc)
    goals = goals.copy()
    goals[2, 1] = np.nan
    gpu = U.gpu_solve(sc.params, ego, obst, goals)
    cost, am = U.gpu_score(sc.params, obst.shape[0], gpu["coef"], sc.meta)
    assert np.isinf(cost[2]) and am != 2
    ok = U.gpu_solve(sc.params, ego, obst, np.delete(goals, 2, axis=0))
    assert np.array_equal(np.delete(gpu["coef"], 2, axis=0), ok["coef"])


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_score_kinds_and_heading_filter(kind):
    sc = scenes.scene_small(11)
    ego, obst, goals = _scene_arrays(sc)
    gpu = U.gpu_solve(sc.params, ego, obst, goals)
    meta = dict(sc.meta); meta["kind"] = kind; meta["w1"] = 1.5; meta["psi_max_deg"] = 4.0
    cg, ag = U.gpu_score(sc.params, obst.shape[0], gpu["coef"], meta)
    co, ao = U.meta_oracle(sc.params, U.f32(gpu["coef"]), meta)
    # same coefficients on both sides: only the FP32 sum differs; the heading
    # decision is compared where |psi| is not within 1e-5 rad of the limit
    _, _, psi = oracle.positions(oracle.params(**sc.params), U.f32(gpu["coef"]))
    near = np.any(np.abs(np.abs(psi) - np.deg2rad(4.0)) < 1e-5, axis=1)
    fin = np.isfinite(co) & ~near
    assert np.array_equal(np.isinf(cg[~near]), np.isinf(co[~near]))
    assert np.all(np.abs(cg[fin] - co[fin]) <= 1e-5 * np.abs(co[fin]) + 1e-4)
    if ao >= 0:
        assert np.isfinite(cg[ag]) and abs(co[ag] - co[ao]) <= 1e-5 * co[ao] + 1e-4
    else:
        assert ag == -1


def test_empty_batch_and_errors():
    import torch

    from paper_2109_10392_gb300 import mmpc
    params = dict(scenes.BASE_PARAMS)
    s = mmpc.Solver(params, 2)
    dev = "cuda:0"
    ego = torch.zeros(4, device=dev); ego[1] = 15
    obst = torch.zeros((2, 4), device=dev)
    goals = torch.zeros((0, 3), device=dev)
    res = s.solve(ego, obst, goals)
    assert res.coef.shape == (0, 36)
    cost, am = s.score(scenes.META_ABS, res.coef)
    torch.cuda.synchronize()
    assert am.item() == -1
    with pytest.raises(mmpc.MmpcError) as ei:
        s.solve(ego, torch.zeros((3, 4), device=dev), torch.zeros((1, 3), device=dev))
    assert ei.value.code == mmpc.MMPC_ERR_SHAPE
    with pytest.raises(mmpc.MmpcError) as ei:
        s.score(dict(scenes.META_ABS, w1=-1.0), torch.zeros((1, 36), device=dev))
    assert ei.value.code == mmpc.MMPC_ERR_INVALID_ARG
    s.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("which", ["small", "large"])
def test_culling_is_exact(which, variant):
    """Culled and dense evaluation of Eq. split_alpha_o give bit-identical
    results; the work counter is exact for the dense path and smaller with
    culling."""
    import torch

    from paper_2109_10392_gb300 import mmpc
    sc = scenes.scene_small(12) if which == "small" else scenes.scene_large(3)
    ego, obst, goals = _scene_arrays(sc)
    out = {}
    for cull in (0, 1):
        params = dict(sc.params, cull=cull, variant=variant)
        s = mmpc.Solver(params, obst.shape[0])
        mmpc.mmpc_take_work_count(s.ctx)
        out[cull] = U.gpu_solve(params, ego, obst, goals, solver=s)
        out[cull]["work"] = mmpc.mmpc_take_work_count(s.ctx)
        s.close()
    for key in ("coef", "lam", "resid", "iters"):
        assert np.array_equal(out[0][key], out[1][key]), key
    B, m, N, K = len(goals), obst.shape[0], sc.params["N"], sc.params["iters"]
    assert out[0]["work"] == B * (K + 1) * m * N
    assert 0 < out[1]["work"] < out[0]["work"]
    torch.cuda.synchronize()


def test_variants_agree():
    """The one-sample and the pair kernels run the same arithmetic per sample
    and differ only in the order of the sums over samples."""
    sc = scenes.scene_small(13)
    ego, obst, goals = _scene_arrays(sc)
    a = U.gpu_solve(dict(sc.params, variant=1), ego, obst, goals)
    b = U.gpu_solve(dict(sc.params, variant=2), ego, obst, goals)
    orc = U.oracle_solve(sc.params, ego, obst, goals)
    sens = U.sensitivity(sc.params, ego, obst, goals, orc["coef"])
    good = sens < U.SENS_TOL
    assert np.all(U.pos_err(sc.params, a["coef"], b["coef"])[good] <= U.POS_TOL)


@pytest.mark.parametrize("iters", [100, 300])
def test_no_drift_over_long_runs(iters):
    """The multiplier update integrates any bias of the per-sample targets, so
    a biased heading sin/cos (or another systematic FP32 error) makes the
    iterate drift away from the oracle linearly in the iteration count.  An
    obstacle-free scene, whose slow heading mode shows such a drift most
    clearly, must stay within the position bar after 300 iterations."""
    sc = scenes.scene_custom(12, 9, 0, N=60, x_range=(-30.0, 120.0))
    params = dict(sc.params)
    params.update(iters=iters, tol=0.0)
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst).reshape(-1, 4), U.f32(sc.goals)
    orc = U.oracle_solve(params, ego, obst, goals)
    for variant in (1, 2):
        params["variant"] = variant
        gpu = U.gpu_solve(params, ego, obst, goals)
        err = U.pos_err(params, gpu["coef"], orc["coef"])
        assert err.max() <= U.POS_TOL, (variant, err)


def test_precision_workload_sampled(capsys):
    """The 16384-goal, 30-obstacle, N = 200, n = 16 workload at its full size,
    FP32 path, 100 iterations: every 256th trajectory against the FP64
    oracle (positions on the conditioning-aware bars, meta costs, the
    argmin over the sample).  Prints the error table."""
    sc = scenes.scene_custom(31, 16384, 30, N=200, n=16)
    params = dict(sc.params)
    params.update(tol=0.0)
    ego, obst, goals = _scene_arrays(sc)
    gpu = U.gpu_solve(params, ego, obst, goals)
    sel = np.arange(0, len(goals), 256)
    orc = U.oracle_solve(params, ego, obst, goals[sel])
    sens = U.sensitivity(params, ego, obst, goals[sel], orc["coef"], trials=1)
    gs = {k: v[sel] for k, v in gpu.items()}
    # The stated bars on the whole parity set.  (The step's K11 u is a
    # compensated dot product: with plain FP32 sums the products, which
    # cancel by five orders of magnitude once the multipliers have grown
    # along K11's near-null directions, cost up to 3.5e-3 m here.)
    err = U.pos_err(params, gs["coef"], orc["coef"])
    good = sens < U.SENS_TOL
    assert good.mean() >= 0.3
    assert np.all(err[good] <= U.POS_TOL), err[good]
    assert np.all(err <= U.CHAOS_TOL), err
    assert np.all(np.isfinite(gs["coef"]))
    meta = dict(sc.meta)
    c_gpu, am_gpu = U.gpu_score(params, obst.shape[0], gs["coef"], meta)
    c_orc, am_orc = U.meta_oracle(params, orc["coef"], meta)
    fin = np.isfinite(c_orc) & np.isfinite(c_gpu)
    rel = np.abs(c_gpu[fin & good] - c_orc[fin & good]) / np.maximum(np.abs(c_orc[fin & good]), 1e-3)
    with capsys.disabled():
        print(f"\n[precision workload, fp32] sample {len(sel)}: parity set {good.mean():.2f}, "
              f"position error max {err[good].max():.2e} median {np.median(err[good]):.2e} m, "
              f"share <= 1e-3 m {np.mean(err[good] <= U.POS_TOL):.3f}; "
              f"all: median {np.median(err):.2e}; meta cost rel error max {rel.max() if rel.size else 0:.2e}; "
              f"argmin gpu {am_gpu} oracle {am_orc}")
    assert rel.size == 0 or rel.max() <= U.COST_RTOL
    # the same argmin over the sample, or an equally good one within the cost tolerance
    assert am_gpu == am_orc or abs(c_orc[am_gpu] - c_orc[am_orc]) <= U.COST_RTOL * abs(c_orc[am_orc])


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("N,n,m,B,iters", [
    (8, 7, 2, 1, 10),       # the smallest horizon, one goal
    (32, 12, 1024, 2, 5),   # the largest obstacle count
    (100, 12, 50, 3, 0),    # no iteration: the cold start itself
])
def test_extreme_shapes(N, n, m, B, iters, variant):
    sc = scenes.scene_custom(seed=N + m + B, B=B, m=m, N=N, n=n, x_range=(-100.0, 400.0))
    params = dict(sc.params)
    params.update(iters=iters, variant=variant, tol=0.0)
    ego, obst, goals = _scene_arrays(sc)
    orc = U.oracle_solve(params, ego, obst, goals)
    gpu = U.gpu_solve(params, ego, obst, goals)
    if iters == 0:
        # the boundary-only QP: well conditioned, no iteration to amplify rounding
        assert np.max(U.pos_err(params, gpu["coef"], orc["coef"])) <= 1e-4
        assert np.all(gpu["iters"] == 0)
    else:
        _check_parity(params, ego, obst, goals, gpu, orc)


def test_step_through_host_memory():
    """mmpc_step_host (copies in, solve, score, copies out) returns exactly what
    the device-buffer calls return; the device buffers it grows are reused."""
    import torch

    from paper_2109_10392_gb300 import mmpc
    sc = scenes.scene_custom(41, 64, 12, N=100)
    params = dict(sc.params)
    m = sc.obst.shape[0]
    meta = mmpc.make_meta(**sc.meta)
    s = mmpc.Solver(params, m)
    n = s.n
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float32)).contiguous()  # noqa: E731
    ego, obst, goals = t(sc.ego), t(sc.obst).reshape(m, 4), t(sc.goals)
    for B in (64, 16, 64):  # grows once, then reuses
        hc = torch.zeros((B, 3 * n)).pin_memory()
        hr = torch.zeros((B, 4)).pin_memory()
        hcost = torch.zeros(B).pin_memory()
        ham = torch.zeros(1, dtype=torch.int32).pin_memory()
        mmpc.mmpc_step_host(s.ctx, meta, ego.pin_memory(), obst.pin_memory(), goals[:B].contiguous().pin_memory(),
                            hc, hcost, ham, hr)
        d = s.solve(ego.cuda(), obst.cuda(), goals[:B].contiguous().cuda(), want_lam=False)
        cost, am = s.score(meta, d.coef)
        torch.cuda.synchronize()
        assert torch.equal(hc, d.coef.cpu()) and torch.equal(hr, d.resid.cpu())
        assert torch.equal(hcost, cost.cpu()) and int(ham.item()) == int(am.item())
        # the same through one contiguous pinned block per direction (one copy each way)
        blk_in = torch.cat([ego.reshape(-1), obst.reshape(-1), goals[:B].reshape(-1)]).pin_memory()
        blk_out = torch.zeros(B * (3 * n + 5)).pin_memory()
        bc = blk_out[:3 * n * B].view(B, 3 * n)
        br = blk_out[3 * n * B:(3 * n + 4) * B].view(B, 4)
        bcost = blk_out[(3 * n + 4) * B:]
        mmpc.mmpc_step_host(s.ctx, meta, blk_in[:4], blk_in[4:4 + 4 * m].view(m, 4), blk_in[4 + 4 * m:].view(B, 3),
                            bc, bcost, ham, br)
        assert torch.equal(bc, hc) and torch.equal(br, hr) and torch.equal(bcost, hcost)
    with pytest.raises(mmpc.MmpcError):
        mmpc.mmpc_step_host(s.ctx, meta, ego, obst[:3].contiguous(), goals, hc, hcost, ham)
    s.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_stall_stop(variant):
    """The opt-in stall stop on a dense scene: (1) a trajectory it stops had,
    at its last check, a residual above stall_tol and above stall_ratio times
    the residual of two checks earlier (both read from fixed-count GPU runs);
    (2) every trajectory that reaches tol without the rule reaches it with the
    rule, at the same iteration, bit for bit; (3) the stopped iterates match the
    oracle run for the same iteration counts (conditioning-aware bar)."""
    sc = scenes.scene_large(0)
    sel = np.arange(0, 1024, 8)
    ego, obst, goals = _scene_arrays(sc)
    goals = goals[sel]
    base = dict(sc.params)
    base.update(tol=1e-2, check_every=10, variant=variant)
    stall = dict(base, stall_tol=1.0, stall_ratio=0.5)
    g0 = U.gpu_solve(base, ego, obst, goals)
    g1 = U.gpu_solve(stall, ego, obst, goals)
    conv0 = np.max(g0["resid"][:, :3], axis=1) <= 1e-2
    conv1 = np.max(g1["resid"][:, :3], axis=1) <= 1e-2
    assert np.all(conv1[conv0])
    assert np.array_equal(g1["coef"][conv0], g0["coef"][conv0]) and np.array_equal(g1["iters"][conv0], g0["iters"][conv0])
    stopped = (g1["iters"] < base["iters"]) & ~conv1
    assert stopped.mean() > 0.3, stopped.mean()  # the dense scene is mostly infeasible
    assert g1["iters"].mean() < 0.75 * g0["iters"].mean()
    fixed = dict(base, tol=0.0)
    for K in np.unique(g1["iters"][stopped]):
        idx = np.where(stopped & (g1["iters"] == K))[0]
        rk = U.gpu_solve(dict(fixed, iters=int(K)), ego, obst, goals[idx])["resid"]
        r2 = U.gpu_solve(dict(fixed, iters=int(K) - 20), ego, obst, goals[idx])["resid"]
        ck, c2 = np.max(rk[:, :3], axis=1), np.max(r2[:, :3], axis=1)
        assert np.all(ck > 1.0) and np.all(ck > 0.5 * c2), (K, ck, c2)
        assert np.array_equal(rk, g1["resid"][idx])
        pk = dict(fixed, iters=int(K))
        orc = U.oracle_solve(pk, ego, obst, goals[idx])
        _check_parity(pk, ego, obst, goals[idx], {"coef": g1["coef"][idx]}, orc, min_frac=0.0)


def test_measured_fp32_peaks_plausible():
    """mmpc_measure_peaks: the saturating FFMA, FFMA2 and rsqrt kernels run
    at rates that the unit counts allow (at most 128 FP32 lanes and 16 MUFU
    units per SM and clock, at the maximum clock, plus timing slack) and
    that are not far below them either."""
    from paper_2109_10392_gb300 import mmpc
    pk = mmpc.mmpc_measure_peaks(reps=2)
    per_clk = lambda v: v / (pk["sms"] * pk["clock_khz"] * 1e3)  # noqa: E731
    assert 48 <= per_clk(pk["ffma"]) <= 128 * 1.05, pk
    assert 48 <= per_clk(pk["ffma2"]) <= 128 * 1.05, pk
    assert 4 <= per_clk(pk["rsqrt"]) <= 16 * 1.05, pk
    with pytest.raises(mmpc.MmpcError):
        mmpc.mmpc_measure_peaks(reps=0)
