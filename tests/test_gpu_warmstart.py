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
