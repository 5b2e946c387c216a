"""Direct pin of the oracle's multiplier step (Sec. III-E, "Multiplier
Update") and of its residual definitions.

One iteration of the oracle is recomputed here in numpy from a basis and an F
built in this file (Bernstein polynomials from binomial coefficients; F_o is
P stacked once per obstacle, then the acceleration block Pddot and the
velocity block Pdot, per axis, as in Eq. aug_cost), starting from the
oracle's own c^{k+1}:

    lambda_xy^{k+1} = lambda_xy^k - rho F^T (F c^{k+1} - g^{k+1})
    lambda_psi^{k+1} = lambda_psi^k - rho P^T (P c_psi^{k+1} - theta^{k+1})

with g^{k+1} from the closed forms of Eqs. split_alpha_o, split_alpha_a and
v_update evaluated at c^{k+1}.  rho is set away from 1 and the starting
multipliers are non-zero, so a dropped rho, a wrong sign, a missing block of
F or a stale g fails here.
"""
import math

import numpy as np
import pytest

from paper_2109_10392_gb300 import scenes


def _basis(N, n, T):
    """Bernstein basis of degree n - 1 on tau = t / T at t_i = i T / (N - 1),
    and its first two time derivatives, from the binomial form."""
    p = n - 1
    tau = np.linspace(0.0, 1.0, N)

    def b(k, deg):
        if k < 0 or k > deg:
            return np.zeros(N)
        return math.comb(deg, k) * tau ** k * (1 - tau) ** (deg - k)

    P = np.stack([b(k, p) for k in range(n)], axis=1)
    Pd = np.stack([p * (b(k - 1, p - 1) - b(k, p - 1)) for k in range(n)], axis=1) / T
    Pdd = np.stack([p * (p - 1) * (b(k - 2, p - 2) - 2 * b(k - 1, p - 2) + b(k, p - 2)) for k in range(n)],
                   axis=1) / T ** 2
    return P, Pd, Pdd


def _targets(c, P, Pd, Pdd, obst, t, prm):
    """g^{k+1} per axis (obstacle blocks, acceleration, velocity) and theta at
    the coefficients c = (c_x, c_y, c_psi)."""
    n = P.shape[1]
    cx, cy, cp = c[:n], c[n:2 * n], c[2 * n:]
    x, y = P @ cx, P @ cy
    xd, yd = Pd @ cx, Pd @ cy
    xdd, ydd = Pdd @ cx, Pdd @ cy
    psi = P @ cp
    a, b = prm["a"], prm["b"]
    gx_o, gy_o = [], []
    for (x0, y0, vx, vy) in obst:
        xi_x, xi_y = x0 + vx * t, y0 + vy * t
        wx, wy = x - xi_x, y - xi_y
        al = np.arctan2(a * wy, b * wx)
        d_unc = (a * wx * np.cos(al) + b * wy * np.sin(al)) / (a ** 2 * np.cos(al) ** 2 + b ** 2 * np.sin(al) ** 2)
        d = np.maximum(1.0, d_unc)
        gx_o.append(xi_x + a * d * np.cos(al))
        gy_o.append(xi_y + b * d * np.sin(al))
    al_a = np.arctan2(ydd, xdd)
    d_a = np.minimum(prm["a_max"], np.hypot(xdd, ydd))
    v = np.clip(np.hypot(xd, yd), prm["v_min"], prm["v_max"])
    gx = np.concatenate(gx_o + [d_a * np.cos(al_a), v * np.cos(psi)])
    gy = np.concatenate(gy_o + [d_a * np.sin(al_a), v * np.sin(psi)])
    theta = np.arctan2(yd, xd)
    return gx, gy, theta


@pytest.mark.parametrize("m,rho,seed", [(0, 2.5, 1), (3, 2.5, 2), (5, 0.4, 3)])
def test_one_iteration_multipliers(orc, m, rho, seed):
    kw = dict(scenes.BASE_PARAMS)
    kw.update(N=30, n=9, T=5.0, rho=rho, iters=1, tol=0.0, check_every=1)
    p = orc.params(**kw)
    N, n, T = kw["N"], kw["n"], kw["T"]
    rng = np.random.default_rng(seed)
    ego = np.array([1.75, 15.0, 0.0, 0.0])
    obst = np.stack([rng.uniform(5, 60, m), rng.choice([-1.75, 1.75, 5.25], m), rng.uniform(5, 15, m),
                     np.zeros(m)], axis=1) if m else np.zeros((0, 4))
    goals = np.array([[5.25, 20.0, 0.0], [-1.75, 12.0, 0.0]])
    lam0 = rng.normal(scale=3.0, size=(len(goals), 3 * n))
    init = orc.solve(orc.params(**dict(kw, iters=0)), ego, obst, goals)["coef"]
    r = orc.solve(p, ego, obst, goals, init=init, init_lam=lam0)
    P, Pd, Pdd = _basis(N, n, T)
    t = np.linspace(0.0, T, N)
    Fa = np.vstack([P] * m + [Pdd, Pd])  # one axis of F (Eq. aug_cost)
    for i in range(len(goals)):
        c1 = r["coef"][i]
        gx, gy, theta = _targets(c1, P, Pd, Pdd, obst, t, kw)
        cx, cy, cp = c1[:n], c1[n:2 * n], c1[2 * n:]
        lam_x = lam0[i, :n] - rho * Fa.T @ (Fa @ cx - gx)
        lam_y = lam0[i, n:2 * n] - rho * Fa.T @ (Fa @ cy - gy)
        lam_p = lam0[i, 2 * n:] - rho * P.T @ (P @ cp - theta)
        want = np.concatenate([lam_x, lam_y, lam_p])
        scale = max(1.0, np.abs(want).max())
        assert np.abs(r["lam"][i] - want).max() <= 1e-9 * scale
        # residual components (reading R13): Euclidean norms of the blocks of F c - g
        ex, ey = Fa @ cx - gx, Fa @ cy - gy
        mo = m * N
        r_obs = math.sqrt(float(ex[:mo] @ ex[:mo] + ey[:mo] @ ey[:mo]))
        r_acc = math.sqrt(float(ex[mo:mo + N] @ ex[mo:mo + N] + ey[mo:mo + N] @ ey[mo:mo + N]))
        r_nh = math.sqrt(float(ex[mo + N:] @ ex[mo + N:] + ey[mo + N:] @ ey[mo + N:]))
        r_psi = float(np.linalg.norm(P @ cp - theta))
        assert np.allclose(r["resid"][i], [r_obs, r_acc, r_nh, r_psi], rtol=1e-9, atol=1e-12)


def test_multiplier_pin_catches_a_wrong_rho(orc):
    """The recomputation distinguishes rho from 1: a run at rho = 1 does not
    satisfy the rho = 2.5 update of the same iterate."""
    kw = dict(scenes.BASE_PARAMS)
    kw.update(N=30, n=9, T=5.0, rho=2.5, iters=1, tol=0.0, check_every=1)
    N, n, T = kw["N"], kw["n"], kw["T"]
    ego = np.array([1.75, 15.0, 0.0, 0.0])
    goals = np.array([[5.25, 20.0, 0.0]])
    init = orc.solve(orc.params(**dict(kw, iters=0)), ego, None, goals)["coef"]
    lam0 = np.full((1, 3 * n), 2.0)
    r1 = orc.solve(orc.params(**dict(kw, rho=1.0)), ego, None, goals, init=init, init_lam=lam0)
    P, Pd, Pdd = _basis(N, n, T)
    t = np.linspace(0.0, T, N)
    Fa = np.vstack([Pdd, Pd])
    c1 = r1["coef"][0]
    gx, _, _ = _targets(c1, P, Pd, Pdd, np.zeros((0, 4)), t, kw)
    lam_x_wrong = lam0[0, :n] - 2.5 * Fa.T @ (Fa @ c1[:n] - gx)
    assert np.abs(r1["lam"][0, :n] - lam_x_wrong).max() > 1e-6
