"""The closed-loop MPC harness (paper_2109_10392_gb300/mpc.py): goal sampling
of Sec. III-F, execution of the chosen plan and control extraction (Sec. II),
and, on the GPU, a closed loop whose every decision is checked against the
FP64 oracle deciding from the same state."""
import numpy as np
import pytest

import parity_utils as U
from paper_2109_10392_gb300 import mmpc, mpc, scenes


def test_goal_sampling_shares():
    rng = np.random.default_rng(0)
    hs = mpc.sample_goals(mpc.MpcConfig(task=mpc.HSRL, goals=20), rng)
    assert hs.shape == (20, 3)
    assert np.sum(hs[:, 0] == scenes.LANES[0]) >= 12  # about 60 % on the right lane
    assert np.all(hs[12:, 1] == 25.0)
    cr = mpc.sample_goals(mpc.MpcConfig(task=mpc.CRUISE, goals=11), rng)
    assert set(cr[:4, 0]) == set(scenes.LANES) and np.all(cr[:4, 1] == 20.0)


def test_basis_rows_match_the_builder():
    params = dict(scenes.BASE_PARAMS)
    buf = mmpc.mmpc_build(mmpc.make_params(**params), 0)
    N, n, T = params["N"], params["n"], params["T"]
    P = buf[N:N + N * n].reshape(N, n)
    Pd = buf[N + N * n:N + 2 * N * n].reshape(N, n)
    Pdd = buf[N + 2 * N * n:N + 3 * N * n].reshape(N, n)
    b = mpc.Basis(T, n)
    for i in (0, 1, 37, N - 1):
        r = b.rows(T * i / (N - 1))
        assert np.allclose(r[0], P[i], atol=1e-13)
        assert np.allclose(r[1], Pd[i], atol=1e-11)
        assert np.allclose(r[2], Pdd[i], atol=1e-9)


def test_execute_straight_run():
    n, T = 12, 8.0
    k = np.arange(n)
    coef = np.concatenate([17.0 * T * k / (n - 1), np.full(n, 1.75), np.zeros(n)])
    st = mpc.execute(coef, mpc.Basis(T, n), 0.1, 2.7)
    assert np.isclose(st["x"], 1.7) and np.isclose(st["y"], 1.75) and np.isclose(st["v"], 17.0)
    assert abs(st["steer"]) < 1e-12 and abs(st["acc_cmd"]) < 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("task", [mpc.CRUISE, mpc.HSRL])
def test_closed_loop_decisions_match_the_oracle(task):
    sc = scenes.scene_small(21)
    cfg = mpc.MpcConfig(task=task, goals=11)
    loop = mpc.ClosedLoop(cfg, sc.ego, sc.obst, seed=3)
    meta = mpc.meta_for(cfg)
    checked = 0
    for _ in range(12):
        ego, obst = loop.ego.copy(), loop.obst.copy()
        state = loop.rng.bit_generator.state
        goals = mpc.sample_goals(cfg, loop.rng)
        loop.rng.bit_generator.state = state  # the loop draws the same goals in its step
        log = loop.step()
        assert np.all(np.isfinite(loop.ego))
        # the oracle decides from the same state and goals
        e, o, g = U.f32(ego), U.f32(obst), U.f32(goals)
        orc = U.oracle_solve(cfg.params, e, o, g)
        co, ao = U.meta_oracle(cfg.params, orc["coef"], meta)
        gpu = U.gpu_solve(cfg.params, e, o, g)
        cg, ag = U.gpu_score(cfg.params, o.shape[0], gpu["coef"], meta)
        assert ag == log.argmin or (log.argmin == 0 and ag < 0)
        if ao >= 0 and np.isfinite(co[ao]):
            # same decision unless the two best costs are within the cost tolerance
            assert ag == ao or abs(co[ag] - co[ao]) <= 2 * U.COST_RTOL * abs(co[ao]) + 2e-3
            checked += 1
    loop.close()
    assert checked >= 6
