"""Pins of the oracle's matrices and QP steps (Sec. III-C, Eqs. lin_solve_xy_1/2,
lin_solve_psi_1/2).

* F is checked against its printed block structure, built here from P alone.
* The Gauss-Jordan inverse is checked against the defining identity.
* Each QP step is checked (i) for the boundary rows A c = b to 1e-9, (ii)
  against a generic dense LU solve (numpy) of the KKT system, and (iii) for
  optimality of the augmented cost itself: its directional derivative along
  every direction of null(A) vanishes.  (iii) evaluates the cost from the
  trajectory samples (sum of squared accelerations, penalty over the stacked
  constraint rows) and never touches the oracle's KKT inverses.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_2109_10392_gb300 import scenes


def _params(orc, **over):
    kw = dict(scenes.BASE_PARAMS)
    kw.update(N=24, n=9, T=4.0)
    kw.update(over)
    return orc.params(**kw)


def test_invert_identity(orc):
    rng = np.random.default_rng(0)
    for dim in (1, 5, 35):
        A = rng.normal(size=(dim, dim)) + dim * np.eye(dim)
        Ai = orc.invert(A)
        assert np.allclose(A @ Ai, np.eye(dim), atol=1e-12)
        assert np.allclose(Ai, np.linalg.inv(A), rtol=1e-12, atol=1e-14)


def test_invert_singular_raises(orc):
    with pytest.raises(RuntimeError):
        orc.invert(np.zeros((3, 3)))


@pytest.mark.parametrize("m", [0, 1, 3])
def test_F_block_structure(orc, m):
    p = _params(orc)
    M = orc.matrices(p, m)
    P, Pd, Pdd = orc.bernstein(p.N, p.n, p.T)
    axis = np.vstack([P] * m + [Pdd, Pd]) if m else np.vstack([Pdd, Pd])
    F = scipy.linalg.block_diag(axis, axis)
    assert M["F"].shape == F.shape
    assert np.array_equal(M["F"], F)
    assert np.allclose(M["Q"], Pdd.T @ Pdd)


def _rand_qp_inputs(p, m, rng):
    R = (m + 2) * p.N
    g = rng.normal(scale=3.0, size=2 * R)
    lam = rng.normal(size=2 * p.n)
    bxy = rng.normal(size=11)
    return g, lam, bxy


def _aug_cost_xy(p, m, c, g, lam):
    """Eq. aug_cost restricted to (c_x, c_y), from samples: 1/2 sum xddot^2 +
    1/2 sum yddot^2 - <lambda, c> + rho/2 ||F c - g||^2 with F c formed row by
    row as obstacle rows (x, y repeated m times), acceleration rows and
    velocity rows."""
    import oracle
    P, Pd, Pdd = oracle.bernstein(p.N, p.n, p.T)
    n = p.n
    cx, cy = c[:n], c[n:]
    cost = 0.5 * np.sum((Pdd @ cx) ** 2) + 0.5 * np.sum((Pdd @ cy) ** 2) - lam @ c
    rows = []
    for ax in (cx, cy):
        rows += [P @ ax] * m + [Pdd @ ax, Pd @ ax]
    Fc = np.concatenate(rows)
    return cost + 0.5 * p.rho * np.sum((Fc - g) ** 2)


@pytest.mark.parametrize("m", [0, 2])
def test_qp_xy_step(orc, m):
    rng = np.random.default_rng(1 + m)
    p = _params(orc)
    g, lam, bxy = _rand_qp_inputs(p, m, rng)
    c, mu = orc.qp_xy(p, m, g, lam, bxy)
    M = orc.matrices(p, m)
    A = M["Axy"]
    # (i) boundary rows
    assert np.max(np.abs(A @ c - bxy)) < 1e-9
    # (ii) generic dense LU solve of the same KKT system
    n2 = 2 * p.n
    Qxy = scipy.linalg.block_diag(M["Q"], M["Q"])
    K = np.block([[Qxy + p.rho * M["F"].T @ M["F"], A.T], [A, np.zeros((11, 11))]])
    sol = np.linalg.solve(K, np.concatenate([p.rho * M["F"].T @ g + lam, bxy]))
    assert np.allclose(c, sol[:n2], rtol=1e-10, atol=1e-10)
    assert np.allclose(mu, sol[n2:], rtol=1e-8, atol=1e-8)
    # (iii) stationarity of the augmented cost on null(A)
    Z = scipy.linalg.null_space(A)
    h = 1e-3
    scale = abs(_aug_cost_xy(p, m, c, g, lam)) + 1.0
    for z in Z.T:
        dd = (_aug_cost_xy(p, m, c + h * z, g, lam) - _aug_cost_xy(p, m, c - h * z, g, lam)) / (2 * h)
        assert abs(dd) < 1e-7 * scale
    # and it is a minimum: any feasible move raises the cost
    f0 = _aug_cost_xy(p, m, c, g, lam)
    for _ in range(5):
        z = Z @ rng.normal(size=Z.shape[1])
        assert _aug_cost_xy(p, m, c + 0.1 * z, g, lam) > f0


def test_qp_psi_step(orc):
    import oracle
    rng = np.random.default_rng(7)
    p = _params(orc)
    theta = rng.normal(scale=0.2, size=p.N)
    lam = rng.normal(size=p.n)
    bpsi = rng.normal(scale=0.1, size=4)
    c, mu = orc.qp_psi(p, theta, lam, bpsi)
    M = orc.matrices(p, 0)
    A = M["Apsi"]
    assert np.max(np.abs(A @ c - bpsi)) < 1e-9
    P, Pd, Pdd = oracle.bernstein(p.N, p.n, p.T)
    K = np.block([[Pdd.T @ Pdd + p.rho * P.T @ P, A.T], [A, np.zeros((4, 4))]])
    sol = np.linalg.solve(K, np.concatenate([p.rho * P.T @ theta + lam, bpsi]))
    assert np.allclose(c, sol[:p.n], rtol=1e-10, atol=1e-10)

    def cost(cc):  # Eq. split_psi, last line: f(c_psi) + rho/2 ||theta - P c_psi||^2
        return 0.5 * np.sum((Pdd @ cc) ** 2) - lam @ cc + 0.5 * p.rho * np.sum((theta - P @ cc) ** 2)
    Z = scipy.linalg.null_space(A)
    for z in Z.T:
        dd = (cost(c + 1e-3 * z) - cost(c - 1e-3 * z)) / 2e-3
        assert abs(dd) < 1e-8 * (abs(cost(c)) + 1)


def test_boundary_values_reading(orc):
    """Boundary vector layout: x rows (x0, xdot0, xddot0, xdot_T, xddot_T), y rows
    (y0, ydot0, yddot0, y_T, ydot_T, yddot_T), psi rows (psi0, psidot0, psi_T,
    psidot_T)."""
    ego = np.array([1.75, 15.0, 0.1, 0.5])
    goal = np.array([-5.25, 25.0, 0.3])
    bxy, bpsi = orc.boundary(ego, goal)
    c, s = np.cos(0.1), np.sin(0.1)
    assert np.allclose(bxy, [0, 15 * c, 0.5 * c, 25.0, 0.3, 1.75, 15 * s, 0.5 * s, -5.25, 0, 0])
    assert np.allclose(bpsi, [0.1, 0, 0, 0])
