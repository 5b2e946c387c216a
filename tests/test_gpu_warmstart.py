"""The learned warm start end to end on the GPU, at a small size: a network
trained by the library's own kernels on scenes solved by the plain method
(coefficients of the trajectories that reached the residual target; the
multipliers lambda^0 = Q c^0) must start converging trajectories closer to
their solutions than the cold start does -- fewer AM iterations to residual
<= 1e-2 m -- and the fallback must re-solve exactly the trajectories the
warm start missed, from the cold start, so that no trajectory converges less
often than without the network."""
import pytest

from paper_2109_10392_gb300 import warmstart

pytestmark = pytest.mark.gpu


def test_warm_start_gains_over_cold_start():
    import torch
    dev = torch.device("cuda:0")
    cfg = warmstart.WarmConfig(train_scenes=30000, goals_per_scene=8, obstacles=10, x_range=(-30.0, 120.0),
                               steps=1500, batch=4096, seed=3)
    X, T = warmstart.build_dataset(cfg, dev)
    ws, losses = warmstart.train(cfg, X, T, dev, log_every=250)
    assert losses[-1][1] < 0.3 * losses[0][1], losses
    r = warmstart.evaluate(ws, cfg, dev, S=128, B=128, reps=1)
    ws.close()
    assert r["warm_fallback"]["fallback_equals_cold"]
    assert r["warm_fallback"]["fallbacks"] == r["warm"]["misses"]
    # the fallback keeps every trajectory the cold start converges
    assert r["warm_fallback"]["converged"] >= r["cold"]["converged"]
    assert r["converged_both"] > 1000, r
    it = r["iters_both_converged"]
    assert it["warm"] < 0.85 * it["cold"], r


def test_budget_only_fallback_with_stall_stop():
    """Fallback mode 2 (not in the paper): with the stall stop on, only the
    warm-started misses that ran the whole iteration budget are solved again
    from the cold start; the stalled ones keep their warm-started result."""
    import torch
    dev = torch.device("cuda:0")
    cfg = warmstart.WarmConfig(train_scenes=20000, goals_per_scene=8, obstacles=50, steps=800, batch=4096, seed=4)
    X, T = warmstart.build_dataset(cfg, dev)
    ws, _ = warmstart.train(cfg, X, T, dev, log_every=400)
    r = warmstart.evaluate(ws, cfg, dev, S=64, B=128, reps=1, stall=(1.0, 0.5))
    ws.close()
    fb2, fb1 = r["warm_fallback_budget"], r["warm_fallback"]
    assert fb2["fallbacks"] == fb2["budget_misses"]
    assert fb1["fallbacks"] == r["warm"]["misses"]
    assert fb2["fallbacks"] <= fb1["fallbacks"]
    assert r["warm"]["converged"] <= fb2["converged"] <= fb1["converged"]
    assert fb2["passes"] <= fb1["passes"]
