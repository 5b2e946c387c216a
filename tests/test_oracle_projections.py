"""Pins of the oracle's closed-form steps (Eqs. v_update, split_alpha_o,
split_alpha_a) against brute-force minimisation on tiny inputs.

* alpha, d (Eq. split_alpha_o with d >= 1): in ellipse-normalised
  coordinates (w_x/a, w_y/b) the printed closed forms are exactly the
  projection onto the exterior of the unit disk, found here by sampling the
  angle on a fine grid; for a = b the same holds in raw coordinates; and the
  unconstrained d equals the normalised distance hypot(w_x/a, w_y/b).
* alpha_a, d_a: the Euclidean projection onto the disk of radius a_max.
* v: the 1-D argmin of the non-holonomic penalty along the velocity
  direction, clipped to [v_min, v_max].
"""
import numpy as np
import pytest

ANG = np.linspace(-np.pi, np.pi, 200001)


def _brute_exterior(u):
    """argmin over (alpha, d >= 1) of |u - d (cos alpha, sin alpha)|^2."""
    dirs = np.stack([np.cos(ANG), np.sin(ANG)], 1)
    d = np.maximum(1.0, dirs @ u)
    pts = d[:, None] * dirs
    k = np.argmin(np.sum((pts - u) ** 2, 1))
    return pts[k]


@pytest.mark.parametrize("a,b", [(5.6, 2.5), (5.6, 3.1), (3.0, 3.0)])
def test_obstacle_projection_matches_brute_force(orc, a, b):
    rng = np.random.default_rng(11)
    for _ in range(40):
        wx, wy = rng.uniform(-15, 15), rng.uniform(-6, 6)
        al, d = orc.project_obstacle(wx, wy, a, b)
        assert d >= 1.0
        target_n = np.array([d * np.cos(al), d * np.sin(al)])  # normalised target
        u = np.array([wx / a, wy / b])
        bf = _brute_exterior(u)
        assert np.allclose(target_n, bf, atol=5e-4 * max(1.0, np.linalg.norm(u)))
        # unconstrained d equals the normalised distance
        assert np.isclose(d, max(1.0, np.hypot(wx / a, wy / b)), rtol=1e-12)
        if a == b:  # raw coordinates: exact Euclidean projection on the disk's exterior
            raw = np.array([a * d * np.cos(al), b * d * np.sin(al)])
            dirs = np.stack([np.cos(ANG), np.sin(ANG)], 1)
            dd = np.maximum(a, dirs @ np.array([wx, wy]))
            pts = dd[:, None] * dirs
            best = pts[np.argmin(np.sum((pts - [wx, wy]) ** 2, 1))]
            assert np.allclose(raw, best, atol=2e-3)


def test_obstacle_projection_outside_is_identity(orc):
    """Outside the ellipse the constraint row is met exactly: target = w."""
    a, b = 5.6, 2.5
    for wx, wy in [(20.0, 0.3), (-7.0, 2.0), (0.0, 3.0), (4.0, -2.2)]:
        al, d = orc.project_obstacle(wx, wy, a, b)
        if np.hypot(wx / a, wy / b) >= 1:
            assert np.allclose([a * d * np.cos(al), b * d * np.sin(al)], [wx, wy], atol=1e-12)


def test_obstacle_projection_degenerate_center(orc):
    al, d = orc.project_obstacle(0.0, 0.0, 5.6, 2.5)
    assert al == 0.0 and d == 1.0


def test_accel_projection_matches_brute_force(orc):
    rng = np.random.default_rng(5)
    amax = 4.0
    dirs = np.stack([np.cos(ANG), np.sin(ANG)], 1)
    for _ in range(40):
        u = rng.uniform(-8, 8, size=2)
        al, da = orc.project_accel(u[0], u[1], amax)
        assert da <= amax + 1e-15
        tgt = da * np.array([np.cos(al), np.sin(al)])
        dd = np.clip(dirs @ u, 0.0, amax)  # d_a is a magnitude: 0 <= d_a <= a_max
        pts = dd[:, None] * dirs
        best = pts[np.argmin(np.sum((pts - u) ** 2, 1))]
        assert np.allclose(tgt, best, atol=2e-4 * max(1, np.linalg.norm(u)))
    al, da = orc.project_accel(0.0, 0.0, amax)
    assert al == 0.0 and da == 0.0


def test_velocity_closed_form(orc):
    rng = np.random.default_rng(3)
    vs = np.linspace(0.1, 30.0, 300001)
    for _ in range(30):
        xd, yd = rng.uniform(-5, 35), rng.uniform(-5, 5)
        th = np.arctan2(yd, xd)
        v = orc.velocity(xd, yd, 0.1, 30.0)
        obj = (xd - vs * np.cos(th)) ** 2 + (yd - vs * np.sin(th)) ** 2
        assert abs(v - vs[np.argmin(obj)]) < 2e-4
        assert 0.1 <= v <= 30.0
