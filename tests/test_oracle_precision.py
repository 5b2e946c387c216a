"""Pins of the oracle's reduced-precision operand emulation: the rounding to
k significant bits agrees with IEEE float32 (k = 24) and with the
independent bfloat16 rounding of the warm-start oracle (k = 8); a hi + lo
pair carries about 2k bits; and on a small scene the position error grows as
the operands lose bits (bfloat16 > TF32 > bfloat16 pair > TF32 pair)."""
import numpy as np

import oracle
from oracle import mlp_oracle
from paper_2109_10392_gb300 import scenes


def test_round_bits_matches_ieee_roundings():
    rng = np.random.default_rng(0)
    x = rng.normal(size=2000) * 10.0 ** rng.uniform(-6, 6, 2000)
    for v in x:
        assert oracle.round_bits(v, 24) == float(np.float32(v))
    xf = x.astype(np.float32)
    for v in xf:
        assert oracle.round_bits(float(v), 8) == mlp_oracle.bf16_round(v)
    assert oracle.round_bits(1 + 2 ** -8, 8) == 1.0          # a tie goes to the even significand
    assert oracle.round_bits(1 + 3 * 2 ** -8, 8) == 1 + 2 ** -6
    assert oracle.round_bits(0.0, 8) == 0.0 and oracle.round_bits(-3.0, 1) == -4.0


def test_split_pairs_carry_twice_the_bits():
    rng = np.random.default_rng(1)
    for v in rng.normal(size=500):
        for k in (8, 11):
            hi = oracle.round_bits(v, k)
            lo = oracle.round_bits(v - hi, k)
            assert abs((hi + lo) - v) <= 2.0 ** (-2 * k + 1) * abs(v)


def test_error_grows_as_operands_lose_bits():
    sc = scenes.scene_custom(5, 6, 3, N=40, n=10, x_range=(-30.0, 120.0))
    kw = dict(sc.params)
    kw.update(tol=0.0, iters=60)
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    exact = oracle.solve(oracle.params(**kw), f(sc.ego), f(sc.obst), f(sc.goals))
    xe, ye, _ = oracle.positions(oracle.params(**kw), exact["coef"])
    err = {}
    for name, bits, split in [("bf16", 8, 0), ("tf32", 11, 0), ("bf16x2", 8, 1), ("tf32x2", 11, 1), ("fp32", 24, 0)]:
        r = oracle.solve(oracle.params(**kw, basis_bits=bits, basis_split=split), f(sc.ego), f(sc.obst), f(sc.goals))
        x, y, _ = oracle.positions(oracle.params(**kw), r["coef"])
        err[name] = float(np.median(np.max(np.hypot(x - xe, y - ye), axis=1)))
    assert err["bf16"] > err["tf32"] > err["bf16x2"] > err["tf32x2"]
    assert err["tf32x2"] < 1e-3 and err["fp32"] < 1e-3 and err["bf16"] > 1e-2
