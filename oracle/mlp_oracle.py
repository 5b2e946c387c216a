"""FP64 oracle of the learned warm start: scene features, the MLP, its
gradients and the AdamW update, and the encoding of solutions as targets.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` import it.  The
CUDA path (``csrc/mmpc_mlp.cu`` behind ``include/mmpc_mlp.h``) shares no code
with it.

The paper gives no learned component; it names learning-based supervision of
the optimizer as the use of its batch solutions (Sec. V).  What is computed
here is therefore the plain definition of each piece, written out in numpy
float64:

* features (61 used, 64 in memory): ego state, the 10 obstacles nearest to the
  ego at t = 0, the goal tuple and a constant 1 (layout in ``features``);
* an MLP 64 -> 256 -> 256 -> 256 -> 6n with GELU (the exact erf form) after
  each hidden layer, weights rounded to bfloat16 (round to nearest even) and
  every product and sum in float64;
* the mean-squared-error loss over standardised targets and its gradients by
  the chain rule (pinned against central finite differences), optionally
  with every operand of every product rounded to bfloat16 as the tensor
  cores take it (``op_bf16``; pinned by a hand-worked one-unit case);
* AdamW with bias correction and decoupled weight decay on the weight
  matrices (Loshchilov & Hutter, "Decoupled Weight Decay Regularization",
  2019);
* targets: a solution (c, lambda) of Algorithm 1 expressed relative to the
  constant-velocity, constant-lane motion of the ego, c_x - v0 lin,
  c_y - y0, c_psi, lambda_x, lambda_y, lambda_psi (lin: the Bernstein
  coefficients of f(t) = t, T k / (n - 1)).

Parity status: every function is pinned by ``tests/test_oracle_mlp.py``
(closed forms, finite differences, hand-built feature cases).
"""
from __future__ import annotations

import math

import numpy as np

FEATURES = 64        # memory width of a feature row
NEAREST = 10         # obstacles in the feature row
SLOT = 5             # features per obstacle
PAD_DX = 10.0        # dx feature of an empty obstacle slot (1000 m ahead)
LANE_WIDTH = 3.5
ROAD_LEFT = 7.0      # lane index = floor((y + 7) / 3.5), clipped to [0, 3]

# feature scales
Y_SCALE, V_SCALE, A_SCALE, X_SCALE = 3.5, 20.0, 4.0, 100.0


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(x)
    return np.where(nan, np.nan, out)


def lane_index(y):
    """clip(floor((y + 7) / 3.5), 0, 3), formed in float32 with one rounding
    per operation: an integer decision, taken in the GPU's precision."""
    f = np.float32
    q = ((np.asarray(y, dtype=np.float32) + f(ROAD_LEFT)).astype(f) / f(LANE_WIDTH)).astype(f)
    return np.clip(np.floor(q), 0, 3).astype(np.float64)


def nearest_order(ego, obst, a, b):
    """Indices of the obstacles by increasing ellipse-normalised distance to
    the ego at t = 0, ties by index.  The keys (x0/a)^2 + ((y0 - y_ego)/b)^2
    are formed in float32, one rounding per operation, as the GPU forms them:
    the order is an integer decision and both sides take it in float32."""
    f = np.float32
    obst = np.asarray(obst, dtype=np.float64).reshape(-1, 4)
    if obst.shape[0] == 0:
        return np.zeros(0, dtype=np.int64)
    ux = (obst[:, 0].astype(f) / f(a)).astype(f)
    uy = ((obst[:, 1].astype(f) - f(ego[0])).astype(f) / f(b)).astype(f)
    key = ((ux * ux).astype(f) + (uy * uy).astype(f)).astype(f)
    return np.lexsort((np.arange(key.size), key.astype(np.float64)))


def features(ego, obst, goals, a, b):
    """Feature rows [B, 64] of one scene (ego [4], obst [m, 4], goals [B, 3]):
      0-3    y0 / 3.5, v0 / 20, psi0, acc0 / 4
      4-53   per slot s (nearest first): x0 / 100, (y0_j - y0) / 3.5,
             (vx_j - v0) / 20, vy_j / 20, lane(y0_j) - lane(y0); an empty
             slot (fewer than 10 obstacles) holds (10, 0, 0, 0, 0)
      54-56  (y_g - y0) / 3.5, v_g / 20, a_g / 4
      57     1
      58-63  0
    """
    ego = np.asarray(ego, dtype=np.float64)
    obst = np.asarray(obst, dtype=np.float64).reshape(-1, 4)
    goals = np.asarray(goals, dtype=np.float64).reshape(-1, 3)
    B = goals.shape[0]
    row = np.zeros(FEATURES)
    row[0:4] = (ego[0] / Y_SCALE, ego[1] / V_SCALE, ego[2], ego[3] / A_SCALE)
    order = nearest_order(ego, obst, a, b)[:NEAREST]
    for s in range(NEAREST):
        o = 4 + SLOT * s
        if s < order.size:
            x0, y0, vx, vy = obst[order[s]]
            row[o:o + SLOT] = (x0 / X_SCALE, (y0 - ego[0]) / Y_SCALE, (vx - ego[1]) / V_SCALE, vy / V_SCALE,
                               lane_index(y0) - lane_index(ego[0]))
        else:
            row[o] = PAD_DX
    row[57] = 1.0
    X = np.tile(row, (B, 1))
    X[:, 54] = (goals[:, 0] - ego[0]) / Y_SCALE
    X[:, 55] = goals[:, 1] / V_SCALE
    X[:, 56] = goals[:, 2] / A_SCALE
    return X


def lin(T, n):
    return T * np.arange(n) / (n - 1)


def encode(coef, lam, ego, T, n, outputs=None):
    """Targets [B, outputs] from a solution: (c_x - v0 lin, c_y - y0, c_psi)
    and, for outputs = 6n, (lambda_x, lambda_y, lambda_psi)."""
    outputs = 6 * n if outputs is None else outputs
    coef = np.asarray(coef, dtype=np.float64).reshape(-1, 3 * n)
    t = coef.copy()
    if outputs == 6 * n:
        t = np.concatenate([t, np.asarray(lam, dtype=np.float64).reshape(-1, 3 * n)], axis=1)
    t[:, :n] -= ego[1] * lin(T, n)
    t[:, n:2 * n] -= ego[0]
    return t


def decode(t, ego, T, n, Q=None):
    """Inverse of `encode`: (coef [B, 3n], lam [B, 3n]).  With 3n outputs
    the multipliers are not predicted: lambda = Q c per axis when Q is given
    (the multipliers of a fixed point of the iteration, whose constraint
    residual F c - g vanishes, up to components in the row space of the
    boundary rows), else 0."""
    t = np.asarray(t, dtype=np.float64)
    t = t.reshape(t.shape[0] if t.ndim > 1 else 1, -1).copy()
    t[:, :n] += ego[1] * lin(T, n)
    t[:, n:2 * n] += ego[0]
    coef = t[:, :3 * n]
    if t.shape[1] == 6 * n:
        return coef, t[:, 3 * n:]
    if Q is None:
        return coef, np.zeros_like(coef)
    Q = np.asarray(Q, dtype=np.float64)
    lam = np.concatenate([coef[:, a * n:(a + 1) * n] @ Q.T for a in range(3)], axis=1)
    return coef, lam


# ---------------------------------------------------------------------------
# MLP
# ---------------------------------------------------------------------------
_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    """x Phi(x), Phi the standard normal CDF (exact erf form)."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx x Phi(x) = Phi(x) + x phi(x)."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(Ws, bs, X, bf16=True, act_bf16=False):
    """Ws[i] [in, out] (float32 master weights), bs[i] [out].  Returns the
    outputs and the cache (inputs of each layer, pre-activations).  With
    act_bf16 every layer's input (the features, then each hidden activation,
    held as float32) is rounded to bfloat16 before its product, as the
    tensor-core path stages it."""
    h = np.asarray(X, dtype=np.float64)
    acts, pres = [h], []
    L = len(Ws)
    for i, (W, b) in enumerate(zip(Ws, bs)):
        Wq = bf16_round(W) if bf16 else np.asarray(W, dtype=np.float64)
        hin = bf16_round(h.astype(np.float32)) if act_bf16 else h
        z = hin @ Wq + np.asarray(b, dtype=np.float64)
        pres.append(z)
        h = gelu(z) if i < L - 1 else z
        if i < L - 1:
            acts.append(h)
    return h, (acts, pres)


def loss_and_grads(Ws, bs, X, Z, bf16=True, op_bf16=False):
    """Mean squared error over all outputs, L = sum (y - Z)^2 / (B * outs),
    and its gradients with respect to every weight matrix and bias (the
    gradient of a bfloat16-rounded weight is passed to its master copy).

    op_bf16: every operand of every matrix product is rounded to bfloat16
    (held as float32 first), as the tensor cores take them -- the layer
    inputs of the forward products (act_bf16), and in the backward pass the
    output gradient d of each layer and that layer's input, in both
    d W^T and H^T d.  The bias gradients sum the unrounded d."""
    y, (acts, pres) = forward(Ws, bs, X, bf16, act_bf16=op_bf16)
    Z = np.asarray(Z, dtype=np.float64)
    cnt = y.size
    r = y - Z
    L = float(np.sum(r * r) / cnt)
    d = 2.0 * r / cnt
    rnd = (lambda a: bf16_round(np.asarray(a).astype(np.float32))) if op_bf16 else (lambda a: a)
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        dq = rnd(d)
        gW[i] = rnd(acts[i]).T @ dq
        gb[i] = d.sum(axis=0)
        if i > 0:
            Wq = bf16_round(Ws[i]) if bf16 else np.asarray(Ws[i], dtype=np.float64)
            d = (dq @ Wq.T) * gelu_grad(pres[i - 1])
    return L, gW, gb


def adamw(w, g, m, v, step, lr, beta1, beta2, eps, wd):
    """One AdamW update of the parameter w with gradient g (step counts from
    1); returns (w, m, v).  wd = 0 for biases."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    w = w - lr * (mh / (np.sqrt(vh) + eps) + wd * w)
    return w, m, v
