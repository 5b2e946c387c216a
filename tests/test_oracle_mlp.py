"""Pins of the warm-start oracle (oracle/mlp_oracle.py) against what the
mathematics fixes: values of the normal CDF, the GELU identities, central
finite differences of the loss, the closed form of the first AdamW steps,
bfloat16 rounding of hand-picked values, hand-built feature rows and the
target encoding of a straight constant-speed run."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_gelu_values_and_identities():
    # Phi(1) = 0.8413447460685429 and Phi(2) = 0.9772498680518208 (normal table)
    assert M.gelu(0.0) == 0.0
    assert abs(M.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(M.gelu(2.0) - 2 * 0.9772498680518208) < 1e-14
    x = np.linspace(-6, 6, 101)
    # x Phi(x) - (-x) Phi(-x) = x (Phi(x) + Phi(-x)) = x
    assert np.allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-14)
    assert abs(M.gelu_grad(0.0) - 0.5) < 1e-15
    # derivative against central differences
    h = 1e-6
    assert np.allclose(M.gelu_grad(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h), atol=1e-8)


def test_bf16_rounding():
    cases = [(1.0, 1.0), (1 + 2 ** -8, 1.0),                 # a tie goes to the even mantissa
             (1 + 3 * 2 ** -8, 1 + 2 ** -6),                 # a tie goes to the even mantissa
             (1 + 2 ** -8 + 2 ** -20, 1 + 2 ** -7),          # above the tie
             (-2.5, -2.5), (0.0, 0.0)]
    for x, want in cases:
        assert M.bf16_round(np.float32(x)) == want, x
    assert np.isnan(M.bf16_round(np.float32(np.nan)))


def _tiny_net(seed=0, sizes=(5, 7, 6, 3)):
    rng = np.random.default_rng(seed)
    Ws = [rng.normal(0, 1 / math.sqrt(i), (i, o)).astype(np.float32) for i, o in zip(sizes[:-1], sizes[1:])]
    bs = [rng.normal(0, 0.1, o).astype(np.float32) for o in sizes[1:]]
    return Ws, bs


def test_forward_closed_form_one_unit():
    W1 = np.array([[2.0]], dtype=np.float32)
    b1 = np.array([-1.0], dtype=np.float32)
    W2 = np.array([[3.0]], dtype=np.float32)
    b2 = np.array([0.5], dtype=np.float32)
    y, _ = M.forward([W1, W2], [b1, b2], np.array([[1.0]]))
    # hidden = gelu(2 - 1) = Phi(1); y = 3 Phi(1) + 0.5
    assert abs(y[0, 0] - (3 * 0.8413447460685429 + 0.5)) < 1e-14


def test_gradients_match_finite_differences():
    Ws, bs = _tiny_net()
    rng = np.random.default_rng(1)
    X = rng.normal(size=(4, 5))
    Z = rng.normal(size=(4, 3))
    W64 = [W.astype(np.float64) for W in Ws]
    b64 = [b.astype(np.float64) for b in bs]
    L, gW, gb = M.loss_and_grads(W64, b64, X, Z, bf16=False)
    h = 1e-6
    for i in range(len(W64)):
        for (r, c) in [(0, 0), (W64[i].shape[0] - 1, W64[i].shape[1] - 1), (1, 1)]:
            Wp = [w.copy() for w in W64]
            Wm = [w.copy() for w in W64]
            Wp[i][r, c] += h
            Wm[i][r, c] -= h
            fd = (M.loss_and_grads(Wp, b64, X, Z, bf16=False)[0] - M.loss_and_grads(Wm, b64, X, Z, bf16=False)[0]) / (2 * h)
            assert abs(fd - gW[i][r, c]) < 1e-7 * max(1.0, abs(fd)), (i, r, c, fd, gW[i][r, c])
        bp = [b.copy() for b in b64]
        bm = [b.copy() for b in b64]
        bp[i][0] += h
        bm[i][0] -= h
        fd = (M.loss_and_grads(W64, bp, X, Z, bf16=False)[0] - M.loss_and_grads(W64, bm, X, Z, bf16=False)[0]) / (2 * h)
        assert abs(fd - gb[i][0]) < 1e-7 * max(1.0, abs(fd))


def test_bf16_forward_uses_rounded_weights():
    Ws, bs = _tiny_net(2)
    X = np.random.default_rng(3).normal(size=(3, 5))
    y16, _ = M.forward(Ws, bs, X, bf16=True)
    y64, _ = M.forward([M.bf16_round(W) for W in Ws], bs, X, bf16=False)
    assert np.array_equal(y16, y64)


def test_adamw_first_two_steps_closed_form():
    w0 = np.array([0.5, -2.0, 3.0])
    g1 = np.array([0.1, -0.2, 0.0])
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.999, 1e-8, 0.1
    w1, m1, v1 = M.adamw(w0, g1, np.zeros(3), np.zeros(3), 1, lr, b1, b2, eps, wd)
    # step 1: m_hat = g, v_hat = g^2
    assert np.allclose(w1, w0 - lr * (g1 / (np.abs(g1) + eps) + wd * w0), atol=1e-15)
    g2 = np.array([0.3, 0.1, -0.4])
    w2, _, _ = M.adamw(w1, g2, m1, v1, 2, lr, b1, b2, eps, wd)
    mh = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    assert np.allclose(w2, w1 - lr * (mh / (np.sqrt(vh) + eps) + wd * w1), atol=1e-15)


def test_features_hand_built_scene():
    a, b = 5.6, 2.5
    ego = np.array([1.75, 15.0, 0.01, 0.5])
    # normalised distances: o0 (x 40, same lane) 7.14; o1 (x -10, lane -1.75) 2.22;
    # o2 (x 5.6, lane 5.25) 1.80; o3 (x -5.6, lane 5.25) 1.80 -> tie with o2, lower index first
    obst = np.array([[40.0, 1.75, 20.0, 0.0], [-10.0, -1.75, 12.0, 0.0], [5.6, 5.25, 16.0, 0.0],
                     [-5.6, 5.25, 18.0, 0.0]])
    goals = np.array([[-1.75, 25.0, 0.0], [5.25, 10.0, 1.0]])
    X = M.features(ego, obst, goals, a, b)
    assert X.shape == (2, 64)
    assert np.allclose(X[0, :4], [0.5, 0.75, 0.01, 0.125])
    order = [2, 3, 1, 0]
    lanes = {0: 2, 1: 1, 2: 3, 3: 3}
    for s, j in enumerate(order):
        x0, y0, vx, vy = obst[j]
        want = [x0 / 100, (y0 - 1.75) / 3.5, (vx - 15.0) / 20, vy / 20, lanes[j] - 2]
        assert np.allclose(X[0, 4 + 5 * s:9 + 5 * s], want), s
    for s in range(4, 10):
        assert np.array_equal(X[0, 4 + 5 * s:9 + 5 * s], [10.0, 0, 0, 0, 0])
    assert np.allclose(X[:, 54:57], [[-1.0, 1.25, 0.0], [1.0, 0.5, 0.25]])
    assert np.all(X[:, 57] == 1.0) and np.all(X[:, 58:] == 0.0)
    assert np.array_equal(X[0, :54], X[1, :54])


def test_features_keep_ten_nearest():
    rng = np.random.default_rng(5)
    ego = np.array([-1.75, 18.0, 0.0, 0.0])
    obst = np.stack([rng.uniform(-50, 250, 30), rng.choice([-5.25, -1.75, 1.75, 5.25], 30),
                     rng.uniform(5, 20, 30), np.zeros(30)], 1)
    X = M.features(ego, obst, np.zeros((1, 3)), 5.6, 2.5)
    d = np.hypot(obst[:, 0] / 5.6, (obst[:, 1] + 1.75) / 2.5)
    want = np.argsort(d, kind="stable")[:10]
    got_x = X[0, 4:54:5] * 100
    assert np.allclose(got_x, obst[want, 0])


def test_encode_straight_run_is_zero_and_round_trip():
    n, T = 12, 8.0
    ego = np.array([1.75, 17.0, 0.0, 0.0])
    coef = np.concatenate([ego[1] * M.lin(T, n), np.full(n, ego[0]), np.zeros(n)])[None]
    lam = np.zeros((1, 3 * n))
    t = M.encode(coef, lam, ego, T, n)
    assert np.allclose(t, 0.0, atol=1e-12)
    rng = np.random.default_rng(0)
    c, l = rng.normal(size=(3, 3 * n)), rng.normal(size=(3, 3 * n))
    c2, l2 = M.decode(M.encode(c, l, ego, T, n), ego, T, n)
    assert np.allclose(c2, c) and np.allclose(l2, l)


def test_lane_index():
    assert list(M.lane_index([-5.25, -1.75, 1.75, 5.25, -9.0, 9.0])) == [0, 1, 2, 3, 0, 3]


@pytest.mark.parametrize("bf16", [False, True])
def test_loss_is_mean_square(bf16):
    Ws, bs = _tiny_net(4)
    X = np.random.default_rng(6).normal(size=(5, 5))
    y, _ = M.forward(Ws, bs, X, bf16)
    L, _, _ = M.loss_and_grads(Ws, bs, X, y + 0.5, bf16)
    assert abs(L - 0.25) < 1e-14


def test_consistent_multipliers_of_a_straight_run_vanish(orc):
    """lambda = Q c with Q = Pdd^T Pdd: a constant-speed, constant-lane run has
    zero second derivative, so its multipliers are 0; and Q c equals
    Pdd^T (Pdd c) computed from the basis directly."""
    from paper_2109_10392_gb300 import scenes
    p = dict(scenes.BASE_PARAMS)
    n, T = p["n"], p["T"]
    Mx = orc.matrices(orc.params(**p), 0)
    Q, Pdd = Mx["Q"], Mx["Pdd"]
    ego = np.array([-1.75, 16.0, 0.0, 0.0])
    c, lam = M.decode(np.zeros((1, 3 * n)), ego, T, n, Q=Q)
    assert np.max(np.abs(lam)) < 1e-9 * np.abs(Q).max() * 16.0 * T
    rng = np.random.default_rng(1)
    t = rng.normal(size=(4, 3 * n))
    c, lam = M.decode(t, ego, T, n, Q=Q)
    for a in range(3):
        want = (Pdd @ c[:, a * n:(a + 1) * n].T).T @ Pdd
        assert np.allclose(lam[:, a * n:(a + 1) * n], want, rtol=1e-10, atol=1e-8)
    c0, lam0 = M.decode(t, ego, T, n)
    assert np.array_equal(c0, c) and np.all(lam0 == 0.0)
    assert M.encode(c, lam, ego, T, n, outputs=3 * n).shape == (4, 3 * n)
    assert np.allclose(M.encode(c, lam, ego, T, n, outputs=3 * n), t)


def test_bf16_activations_round_every_layer_input():
    """act_bf16: the result equals the plain forward of a network whose every
    layer input is replaced by its bfloat16 rounding (built layer by layer)."""
    Ws, bs = _tiny_net(8)
    X = np.random.default_rng(9).normal(size=(6, 5))
    y, _ = M.forward(Ws, bs, X, bf16=True, act_bf16=True)
    h = X
    for i, (W, b) in enumerate(zip(Ws, bs)):
        z = M.bf16_round(h.astype(np.float32)) @ M.bf16_round(W) + b.astype(np.float64)
        h = M.gelu(z) if i < len(Ws) - 1 else z
    assert np.array_equal(y, h)
    y0, _ = M.forward(Ws, bs, X, bf16=True)
    assert 0 < np.max(np.abs(y - y0)) < 0.05 * np.abs(y0).max()


def test_bf16_operand_gradients_hand_case():
    """op_bf16 on a 1 -> 1 -> 1 network worked by hand: the input 1 + 2^-9
    rounds to 1, the output gelu(1) = 0.84134... to 0.83984375 (215 / 256),
    the output gradient 2 y = 1.6796875 is exact in bfloat16, the hidden
    gradient 2 y gelu'(1) = 1.81961... rounds to 1.8203125 (233 / 128) for
    the weight gradient while the bias gradient keeps it unrounded."""
    Ws = [np.array([[1.0]], dtype=np.float32), np.array([[1.0]], dtype=np.float32)]
    bs = [np.zeros(1, dtype=np.float32), np.zeros(1, dtype=np.float32)]
    X = np.array([[1.0 + 2.0 ** -9]])
    Z = np.zeros((1, 1))
    L, gW, gb = M.loss_and_grads(Ws, bs, X, Z, bf16=True, op_bf16=True)
    y = 215.0 / 256.0
    assert L == y * y
    d1 = 2.0 * y
    assert gb[1][0] == d1 and gW[1][0, 0] == y * d1
    phi1 = 0.5 * (1.0 + math.erf(1.0 / math.sqrt(2.0)))
    dens1 = math.exp(-0.5) / math.sqrt(2.0 * math.pi)
    d0 = d1 * (phi1 + dens1)
    assert abs(d0 - 1.8196) < 1e-4
    assert abs(gb[0][0] - d0) < 1e-15
    assert gW[0][0, 0] == 233.0 / 128.0
    # without the operand rounding: y = gelu(x) at the exact input x, and
    # gW0 = x * 2 y gelu'(x)
    x = 1.0 + 2.0 ** -9
    _, gW2, _ = M.loss_and_grads(Ws, bs, X, Z, bf16=True)
    yx = x * 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))
    gx = 0.5 * (1.0 + math.erf(x / math.sqrt(2.0))) + x * math.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    assert abs(gW2[0][0, 0] - x * 2.0 * yx * gx) < 1e-14


def test_bf16_operand_gradients_near_the_plain_ones():
    """The roundings move every gradient by a bfloat16-sized relative amount
    (nonzero, well under 5 %) on a random network; the loss moves only by the
    rounding of the forward inputs."""
    Ws, bs = _tiny_net(11)
    rng = np.random.default_rng(12)
    X = rng.normal(size=(40, 5))
    Z = rng.normal(size=(40, Ws[-1].shape[1]))
    L0, gW0, gb0 = M.loss_and_grads(Ws, bs, X, Z, bf16=True)
    L1, gW1, gb1 = M.loss_and_grads(Ws, bs, X, Z, bf16=True, op_bf16=True)
    assert 0 < abs(L1 - L0) < 1e-2 * L0
    for a, b in zip(gW0 + gb0, gW1 + gb1):
        rel = np.abs(a - b).max() / np.abs(a).max()
        assert 0 < rel < 5e-2, rel
