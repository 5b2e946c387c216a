"""Pins of the oracle's full iteration (Algorithm 1, Sec. III-E) by
invariants that hold exactly in the mathematics:

* fixed point: a straight constant-speed run along the ego's lane with no
  obstacles is met by the cold start and kept by every iteration, with all
  residuals zero;
* every iterate satisfies the boundary rows A c = b;
* mirror symmetry y -> -y, lateral translation y -> y + dy, batch
  permutation, obstacle permutation;
* far obstacles give a zero obstacle residual (to rounding);
* residuals shrink on obstacle-free scenes (Sec. IV, "Optimizer
  Convergence"); the heading multiplier with the printed sign diverges there
  while the sign of the xy update converges (the reading taken).
"""
import numpy as np
import pytest

from paper_2109_10392_gb300 import scenes


def _p(orc, **over):
    kw = dict(scenes.BASE_PARAMS)
    kw.update(N=40, n=10, iters=30)
    kw.update(over)
    return orc.params(**kw)


def _scene(seed=0, m=4, B=6):
    rng = np.random.default_rng(seed)
    ego = np.array([-1.75, 14.0, 0.0, 0.0])
    obst = np.stack([rng.uniform(10, 80, m), rng.choice(scenes.LANES, m), rng.uniform(5, 15, m), np.zeros(m)], 1)
    goals = np.stack([rng.choice(scenes.LANES, B), rng.uniform(10, 25, B), np.zeros(B)], 1)
    return ego, obst, goals


def test_straight_run_is_a_fixed_point(orc):
    p = _p(orc, iters=20)
    ego = np.array([1.75, 17.0, 0.0, 0.0])
    goals = np.array([[1.75, 17.0, 0.0]])
    r = orc.solve(p, ego, np.zeros((0, 4)), goals, trace=True)
    x, y, psi = orc.positions(p, r["coef"])
    t = p.T * np.arange(p.N) / (p.N - 1)
    assert np.allclose(x[0], 17.0 * t, atol=1e-9)
    assert np.allclose(y[0], 1.75, atol=1e-9)
    assert np.allclose(psi[0], 0.0, atol=1e-12)
    assert np.max(np.abs(r["trace"])) < 1e-9
    assert np.allclose(r["lam"], 0.0, atol=1e-9)


def test_boundary_rows_hold_after_iterations(orc):
    p = _p(orc)
    ego, obst, goals = _scene(1)
    r = orc.solve(p, ego, obst, goals)
    M = orc.matrices(p, obst.shape[0])
    n = p.n
    for l in range(goals.shape[0]):
        bxy, bpsi = orc.boundary(ego, goals[l])
        c = r["coef"][l]
        assert np.max(np.abs(M["Axy"] @ c[:2 * n] - bxy)) < 1e-9
        assert np.max(np.abs(M["Apsi"] @ c[2 * n:] - bpsi)) < 1e-9


def test_mirror_symmetry(orc):
    p = _p(orc)
    ego, obst, goals = _scene(2)
    r1 = orc.solve(p, ego, obst, goals)
    e2 = ego.copy(); e2[0] *= -1; e2[2] *= -1
    o2 = obst.copy(); o2[:, 1] *= -1; o2[:, 3] *= -1
    g2 = goals.copy(); g2[:, 0] *= -1
    r2 = orc.solve(p, e2, o2, g2)
    n = p.n
    c1, c2 = r1["coef"], r2["coef"]
    assert np.allclose(c1[:, :n], c2[:, :n], atol=1e-9)
    assert np.allclose(c1[:, n:2 * n], -c2[:, n:2 * n], atol=1e-9)
    assert np.allclose(c1[:, 2 * n:], -c2[:, 2 * n:], atol=1e-9)


def test_lateral_translation(orc):
    p = _p(orc)
    ego, obst, goals = _scene(3)
    dy = 2.3
    r1 = orc.solve(p, ego, obst, goals)
    e2 = ego.copy(); e2[0] += dy
    o2 = obst.copy(); o2[:, 1] += dy
    g2 = goals.copy(); g2[:, 0] += dy
    r2 = orc.solve(p, e2, o2, g2)
    n = p.n
    assert np.allclose(r1["coef"][:, :n], r2["coef"][:, :n], atol=1e-8)
    assert np.allclose(r1["coef"][:, n:2 * n] + dy, r2["coef"][:, n:2 * n], atol=1e-8)
    assert np.allclose(r1["coef"][:, 2 * n:], r2["coef"][:, 2 * n:], atol=1e-9)


def test_batch_and_obstacle_permutation(orc):
    p = _p(orc)
    ego, obst, goals = _scene(4, m=5, B=7)
    r1 = orc.solve(p, ego, obst, goals)
    perm = np.random.default_rng(0).permutation(goals.shape[0])
    r2 = orc.solve(p, ego, obst, goals[perm])
    assert np.array_equal(r1["coef"][perm], r2["coef"])
    operm = np.random.default_rng(1).permutation(obst.shape[0])
    r3 = orc.solve(p, ego, obst[operm], goals)
    assert np.allclose(r1["coef"], r3["coef"], atol=1e-8)


def test_far_obstacles_zero_obstacle_residual(orc):
    p = _p(orc)
    ego, _, goals = _scene(5)
    obst = np.array([[5000.0, 1.75, 10.0, 0.0], [-4000.0, -5.25, 12.0, 0.0]])
    r = orc.solve(p, ego, obst, goals, trace=True)
    # zero up to the rounding of the polar round trip at |xi| ~ 5e3 m
    assert np.all(r["trace"][:, :, 0] < 1e-9)


def test_residuals_shrink_without_obstacles(orc):
    p = _p(orc, N=100, n=12, iters=100)
    ego = np.array([-1.75, 15.0, 0.0, 0.0])
    goals = np.array([(y, v, 0.0) for y in scenes.LANES for v in (15.0, 20.0, 25.0)])
    r = orc.solve(p, ego, np.zeros((0, 4)), goals, trace=True)
    tr = r["trace"]
    conv = np.max(tr[:, :, :3], axis=2)
    assert np.all(conv[:, 100] < 0.05 * conv[:, 0] + 1e-12)
    assert np.all(tr[:, 100, 3] < 0.05 * tr[:, 0, 3] + 1e-12)
    assert np.median(conv[:, 100]) < 1e-2


def test_printed_heading_multiplier_sign_diverges(orc):
    ego = np.array([-1.75, 15.0, 0.0, 0.0])
    goals = np.array([[1.75, 20.0, 0.0], [-5.25, 12.0, 0.0]])
    ok = orc.solve(_p(orc, psi_sign_printed=0, iters=60), ego, np.zeros((0, 4)), goals, trace=True)["trace"]
    bad = orc.solve(_p(orc, psi_sign_printed=1, iters=60), ego, np.zeros((0, 4)), goals, trace=True)["trace"]
    assert np.all(ok[:, -1, 3] < ok[:, 0, 3])
    assert np.all(bad[:, -1, 3] > 10 * bad[:, 0, 3])


def test_early_exit_respects_tolerance(orc):
    p = _p(orc, iters=100, tol=1e-2, check_every=5)
    ego = np.array([-1.75, 15.0, 0.0, 0.0])
    goals = np.array([[-1.75, 16.0, 0.0], [1.75, 18.0, 0.0]])
    r = orc.solve(p, ego, np.zeros((0, 4)), goals)
    for l in range(2):
        k = r["iters"][l]
        assert k % 5 == 0 or k == 100
        if k < 100:
            assert np.max(r["resid"][l, :3]) <= 1e-2
    # the same iteration count run without early exit gives the same result
    p2 = _p(orc, iters=int(r["iters"][0]))
    r2 = orc.solve(p2, ego, np.zeros((0, 4)), goals[:1])
    assert np.array_equal(r2["coef"][0], r["coef"][0])


def test_warm_start_from_own_solution_keeps_it(orc):
    """Restarting from a converged iterate with its multipliers continues the
    same sequence: one more iteration from (c^k, lambda^k) equals c^{k+1}."""
    p10 = _p(orc, iters=10)
    p11 = _p(orc, iters=11)
    p1 = _p(orc, iters=1)
    ego, obst, goals = _scene(6)
    r10 = orc.solve(p10, ego, obst, goals)
    r11 = orc.solve(p11, ego, obst, goals)
    r = orc.solve(p1, ego, obst, goals, init=r10["coef"], init_lam=r10["lam"])
    assert np.allclose(r["coef"], r11["coef"], atol=1e-9)


def test_bad_arguments(orc):
    with pytest.raises(RuntimeError):
        orc.solve(_p(orc, v_min=0.0), np.zeros(4), np.zeros((0, 4)), np.zeros((1, 3)))
    with pytest.raises(RuntimeError):
        orc.solve(_p(orc, n=6), np.zeros(4), np.zeros((0, 4)), np.zeros((1, 3)))
