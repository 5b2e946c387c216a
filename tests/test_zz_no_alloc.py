"""The allocation-free scoring entry point (mmpc_score_static).

It exists for callers that cannot allocate device memory while they run (a
real-time control loop that reserves everything at start-up, or a framework
that only hands out memory from its own pool).  It must give the same costs
and argmin as mmpc_score, call after call, although its scratch is a
library-wide device array that keeps the previous call's contents.  This file
is collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import parity_utils as U
from paper_2109_10392_gb300 import mmpc, scenes

pytestmark = pytest.mark.gpu


def _basis(params):
    import torch
    p = mmpc.make_params(**params)
    buf = mmpc.mmpc_build(p, 0)
    N, n = p.N, p.n
    P = buf[N:N + N * n].reshape(N, n)
    Pd = buf[N + N * n:N + 2 * N * n].reshape(N, n)
    t = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda:0")  # noqa: E731
    return t(P), t(Pd)


def _static(meta, params, P, Pd, coef):
    import torch
    B = coef.shape[0]
    cost = torch.full((B,), -1.0, device="cuda:0")
    am = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
    mmpc.mmpc_score_static(mmpc.make_meta(**meta), params["N"], params["n"], P, Pd, coef, cost, am)
    torch.cuda.synchronize()
    return cost.cpu().numpy(), int(am.item())


# the three meta-cost kinds (cruise, high-speed right lane, absolute), and one
# heading limit tight enough that some trajectories are rejected (+inf)
METAS = {
    "cruise": dict(kind=0, w1=1.0, w2=0.0, v_ref=18.0, y_ref=0.0, psi_max_deg=13.0),
    "hsrl": dict(kind=1, w1=1.0, w2=0.5, v_ref=30.0, y_ref=-5.25, psi_max_deg=13.0),
    "abs": dict(scenes.META_ABS),
    "abs_tight_heading": dict(scenes.META_ABS, psi_max_deg=0.5),
}


@pytest.mark.parametrize("n", [12, 16])
@pytest.mark.parametrize("kind", sorted(METAS))
def test_static_score_matches_context_score(n, kind):
    import torch
    meta = METAS[kind]
    sc = scenes.scene_custom(seed=5, B=3000, m=6, N=100, n=n, x_range=(10.0, 150.0))
    params = dict(sc.params); params["iters"] = 20
    ego, obst, goals = U.f32(sc.ego), U.f32(sc.obst), U.f32(sc.goals)
    s = mmpc.Solver(params, obst.shape[0])
    dev = "cuda:0"
    res = s.solve(torch.tensor(ego, dtype=torch.float32, device=dev),
                  torch.tensor(obst, dtype=torch.float32, device=dev),
                  torch.tensor(goals, dtype=torch.float32, device=dev))
    ref_cost, ref_am = s.score(meta, res.coef)
    torch.cuda.synchronize()
    ref_cost, ref_am = ref_cost.cpu().numpy(), int(ref_am.item())
    if kind == "abs_tight_heading":
        # the case exercises the rejection path on some but not all trajectories
        assert 0 < int(np.isinf(ref_cost).sum()) < len(ref_cost)
    P, Pd = _basis(params)
    for _ in range(2):  # two calls in a row share the scratch array
        cost, am = _static(meta, params, P, Pd, res.coef)
        assert np.array_equal(np.isinf(cost), np.isinf(ref_cost))
        fin = np.isfinite(ref_cost)
        assert np.allclose(cost[fin], ref_cost[fin], rtol=1e-6, atol=1e-6, equal_nan=False)
        assert am == ref_am
    # a different batch after those calls: the previous contents do not leak
    sub = res.coef[:37].contiguous()
    ref2_cost, ref2_am = s.score(meta, sub)
    torch.cuda.synchronize()
    ref2_cost = ref2_cost.cpu().numpy()
    cost, am = _static(meta, params, P, Pd, sub)
    assert np.array_equal(np.isinf(cost), np.isinf(ref2_cost))
    fin = np.isfinite(ref2_cost)
    assert np.allclose(cost[fin], ref2_cost[fin], rtol=1e-6, atol=1e-6)
    assert am == int(ref2_am.item())
    s.close()


def test_static_score_limits():
    import torch
    params = dict(scenes.BASE_PARAMS)
    P, Pd = _basis(params)
    dev = "cuda:0"
    too_many = torch.zeros((mmpc.MMPC_STATIC_SCORE_MAX_B + 1, 36), device=dev)
    cost = torch.empty((too_many.shape[0],), device=dev)
    am = torch.empty((1,), dtype=torch.int32, device=dev)
    with pytest.raises(mmpc.MmpcError) as ei:
        mmpc.mmpc_score_static(mmpc.make_meta(**scenes.META_ABS), 100, 12, P, Pd, too_many, cost, am)
    assert ei.value.code == mmpc.MMPC_ERR_SHAPE
    empty = torch.zeros((0, 36), device=dev)
    mmpc.mmpc_score_static(mmpc.make_meta(**scenes.META_ABS), 100, 12, P, Pd, empty, cost[:0], am)
    torch.cuda.synchronize()
    assert int(am.item()) == -1
