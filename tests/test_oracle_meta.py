"""Pins of the oracle's meta costs (Sec. III-F, Eqs. cruise_cost and
hsrl_cost), the heading restriction (Sec. III assumption 2) and the argmin,
on trajectories whose costs are known in closed form: a straight run x = x0 +
v t, y = y0 has v(t) = v and y(t) = y0 at every one of the N samples."""
import numpy as np

from paper_2109_10392_gb300 import scenes


def _p(orc):
    return orc.params(**scenes.BASE_PARAMS)


def _straight(p, v, y0, psi=0.0):
    n = p.n
    k = np.arange(n)
    return np.concatenate([v * p.T * k / (n - 1), np.full(n, y0), np.full(n, psi)])


def test_closed_form_costs(orc):
    p = _p(orc)
    N = p.N
    coef = np.stack([_straight(p, 18.0, 1.75), _straight(p, 22.5, -5.25)])
    c0, _ = orc.meta_cost(p, coef, kind=orc.META_CRUISE, v_ref=20.0)
    assert np.allclose(c0, [N * 4.0, N * 6.25], rtol=1e-12)
    c1, _ = orc.meta_cost(p, coef, kind=orc.META_HSRL, w1=2.0, w2=0.5, v_ref=30.0, y_ref=-5.25)
    assert np.allclose(c1, [N * (2 * 144 + 0.5 * 49), N * (2 * 56.25)], rtol=1e-12)
    c2, am = orc.meta_cost(p, coef, kind=orc.META_ABS, w1=1.0, w2=0.25, v_ref=20.0, y_ref=-5.25)
    assert np.allclose(c2, [N * (2 + 0.25 * 7), N * 2.5], rtol=1e-12)
    assert am == 1


def test_heading_restriction(orc):
    p = _p(orc)
    coef = np.stack([_straight(p, 20.0, 0.0, np.deg2rad(14.0)), _straight(p, 25.0, 0.0, np.deg2rad(12.0))])
    cost, am = orc.meta_cost(p, coef, kind=orc.META_CRUISE, v_ref=20.0, psi_max=np.deg2rad(13.0))
    assert np.isinf(cost[0]) and np.isfinite(cost[1]) and am == 1
    cost, am = orc.meta_cost(p, coef, kind=orc.META_CRUISE, v_ref=20.0, psi_max=0.0)
    assert np.isfinite(cost).all() and am == 0


def test_argmin_ties_nan_and_empty(orc):
    p = _p(orc)
    a = _straight(p, 21.0, 0.0)
    b = a.copy(); b[0] = np.nan
    coef = np.stack([b, a, a])
    cost, am = orc.meta_cost(p, coef, kind=orc.META_CRUISE, v_ref=20.0)
    assert np.isinf(cost[0]) and am == 1
    cost, am = orc.meta_cost(p, coef[:1], kind=orc.META_CRUISE, v_ref=20.0)
    assert am == -1
    cost, am = orc.meta_cost(p, np.zeros((0, 3 * p.n)), kind=orc.META_CRUISE)
    assert am == -1 and cost.size == 0
