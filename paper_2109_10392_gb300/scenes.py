"""Seeded synthetic highway scenes and workload presets.

This module holds the inputs of the batch trajectory optimizer and nothing of
its arithmetic: random draws of the ego state, the obstacle vehicles and the
goal tuples, plus the named workload presets.  Both the CUDA path's tests and
benchmarks and the FP64 oracle read their inputs from here.

The scenes stand in for the paper's IDM and NGSIM traffic (Sec. IV,
"Implementation Details"), which are not available: a straight 4-lane highway
in the road-attached frame (Sec. III assumption 1), lane width 3.5 m, lane
centres y in {-5.25, -1.75, 1.75, 5.25} m (y positive to the left), obstacle
vehicles moving parallel to the centre line at constant velocity (Sec. III
assumption 3).

Layouts (all float64 here; the CUDA binding casts to float32):
  ego   [4]     y0, v0, psi0, acc0   (x0 = 0 by convention)
  obst  [m, 4]  x0, y0, vx, vy at t = 0
  goals [B, 3]  y_g, v_g, a_g at the end of the horizon
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LANE_WIDTH = 3.5
LANES = np.array([-5.25, -1.75, 1.75, 5.25])

# Physical and solver parameters shared by the workloads.  v_min, v_max,
# a_max and rho are not given in the paper (Eq. v_bound; Sec. III-E); the
# values here are this implementation's choices.
BASE_PARAMS = dict(
    T=8.0,           # horizon [s]
    N=100,           # samples
    n=12,            # Bernstein coefficients per axis (11th order)
    rho=1.0,         # penalty rho_xy
    a=5.6, b=2.5,    # ellipse semi-axes incl. inflation [m]
    v_min=0.1, v_max=30.0, a_max=4.0,
    iters=100,
    tol=0.0,
    check_every=10,
)

META_ABS = dict(kind=2, w1=1.0, w2=0.25, v_ref=20.0, y_ref=-5.25, psi_max_deg=13.0)


@dataclass
class Scene:
    ego: np.ndarray
    obst: np.ndarray
    goals: np.ndarray
    params: dict = field(default_factory=dict)
    meta: dict = field(default_factory=dict)
    name: str = ""
    seed: int = 0


def _spawn_obstacles(rng, m, x_lo, x_hi, v_lo, v_hi, ego_y, a, b, clearance=1.2):
    """m obstacles on random lanes; an obstacle whose ellipse-normalised
    distance to the ego at t = 0 is below `clearance` is drawn again."""
    out = np.zeros((m, 4))
    for j in range(m):
        while True:
            x0 = rng.uniform(x_lo, x_hi)
            y0 = LANES[rng.integers(0, 4)]
            if np.hypot(x0 / a, (y0 - ego_y) / b) >= clearance:
                break
        out[j] = (x0, y0, rng.uniform(v_lo, v_hi), 0.0)
    return out


def scene_small(seed: int = 0, m: int = 10, B: int = 11) -> Scene:
    """One scene, 10 obstacles x ~ U(-30, 120) m, v ~ U(5, 20) m/s; ego on a
    random lane centre with v ~ U(10, 20) m/s; B = 11 goals = the first 11 of
    (lane right to left) x (speed 15, 20, 25 m/s), zero terminal acceleration."""
    rng = np.random.default_rng(seed)
    p = dict(BASE_PARAMS)
    ego_y = LANES[rng.integers(0, 4)]
    ego = np.array([ego_y, rng.uniform(10.0, 20.0), 0.0, 0.0])
    obst = _spawn_obstacles(rng, m, -30.0, 120.0, 5.0, 20.0, ego_y, p["a"], p["b"])
    goals = np.array([(y, v, 0.0) for y in LANES for v in (15.0, 20.0, 25.0)])[:B]
    return Scene(ego, obst, goals, p, dict(META_ABS), f"highway_B{B}_m{m}", seed)


def scene_large(seed: int = 0, m: int = 50, n_offsets: int = 8, n_speeds: int = 128) -> Scene:
    """One scene, 50 obstacles x ~ U(-50, 250) m, v ~ U(5, 20) m/s; B = 1024
    goals = 8 lateral offsets linspace(-5.25, 5.25, 8) x 128 speeds ~ U(5, 30)
    m/s (offset-major), zero terminal acceleration."""
    rng = np.random.default_rng(seed)
    p = dict(BASE_PARAMS)
    ego_y = LANES[rng.integers(0, 4)]
    ego = np.array([ego_y, rng.uniform(10.0, 20.0), 0.0, 0.0])
    obst = _spawn_obstacles(rng, m, -50.0, 250.0, 5.0, 20.0, ego_y, p["a"], p["b"])
    offs = np.linspace(-5.25, 5.25, n_offsets)
    speeds = rng.uniform(5.0, 30.0, size=n_speeds)
    goals = np.array([(y, v, 0.0) for y in offs for v in speeds])
    return Scene(ego, obst, goals, p, dict(META_ABS), f"highway_B{len(goals)}_m{m}", seed)


def scene_custom(seed: int, B: int, m: int, N: int = 100, n: int = 12, x_range=(-50.0, 250.0)) -> Scene:
    """A scene of the large-scene distribution with arbitrary B, m, N, n
    (goals: random lateral offsets in [-5.25, 5.25] m and speeds U(5, 30))."""
    rng = np.random.default_rng(seed)
    p = dict(BASE_PARAMS)
    p["N"] = N
    p["n"] = n
    ego_y = LANES[rng.integers(0, 4)]
    ego = np.array([ego_y, rng.uniform(10.0, 20.0), 0.0, 0.0])
    obst = _spawn_obstacles(rng, m, x_range[0], x_range[1], 5.0, 20.0, ego_y, p["a"], p["b"])
    goals = np.stack([rng.uniform(-5.25, 5.25, B), rng.uniform(5.0, 30.0, B), np.zeros(B)], axis=1)
    return Scene(ego, obst, goals, p, dict(META_ABS), f"highway_B{B}_m{m}_N{N}_n{n}", seed)


def scene_batch(seed: int, S: int = 256, B_range=(16, 512), m_range=(5, 40), N_choices=(50, 100, 150),
                n: int = 12) -> list:
    """S independent scenes of the large-scene distribution with uneven goal
    counts B ~ U{B_range}, obstacle counts m ~ U{m_range} and horizons sampled
    at N in N_choices (the batching workload); scene i has seed (seed, i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(S):
        B = int(rng.integers(B_range[0], B_range[1] + 1))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        N = int(rng.choice(N_choices))
        sub = int(rng.integers(0, 2**31 - 1))
        out.append(scene_custom(sub, B, m, N=N, n=n))
    return out


WARM_WIDTHS = (64, 256, 256, 256, 72)  # warm-start network: features -> 3 x 256 -> 6n (n = 12)


def mlp_init(seed: int, widths=WARM_WIDTHS):
    """Seeded initial weights of an MLP (Glorot-uniform matrices [in, out],
    zero biases), float32.  Random draws only; the network itself is in the
    library."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for i, o in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / (i + o))
        Ws.append(rng.uniform(-lim, lim, (i, o)).astype(np.float32))
        bs.append(np.zeros(o, dtype=np.float32))
    return Ws, bs


def scene_stack(seed: int, S: int, B: int, m: int = 50, x_range=(-50.0, 250.0), goals: str = "random",
                clearance: float = 1.2):
    """S scenes of one shape as stacked float64 arrays (ego [S, 4], obst
    [S, m, 4], goals [S, B, 3]), drawn like `scene_custom` but vectorised:
    ego on a random lane centre with v0 ~ U(10, 20); obstacles on random lanes
    with x ~ U(x_range), vx ~ U(5, 20), redrawn while closer to the ego than
    `clearance` (ellipse-normalised, t = 0).  Goals: "random" draws lateral
    offsets from the 8 offsets linspace(-5.25, 5.25, 8) and speeds ~ U(5, 30);
    "grid" crosses the 8 offsets with B / 8 speeds ~ U(5, 30).  Zero terminal
    acceleration."""
    rng = np.random.default_rng(seed)
    a, b = BASE_PARAMS["a"], BASE_PARAMS["b"]
    ego = np.zeros((S, 4))
    ego[:, 0] = LANES[rng.integers(0, 4, S)]
    ego[:, 1] = rng.uniform(10.0, 20.0, S)
    obst = np.zeros((S, m, 4))
    obst[:, :, 0] = rng.uniform(x_range[0], x_range[1], (S, m))
    obst[:, :, 1] = LANES[rng.integers(0, 4, (S, m))]
    obst[:, :, 2] = rng.uniform(5.0, 20.0, (S, m))
    for _ in range(1000):
        bad = np.hypot(obst[:, :, 0] / a, (obst[:, :, 1] - ego[:, None, 0]) / b) < clearance
        k = int(bad.sum())
        if k == 0:
            break
        obst[:, :, 0][bad] = rng.uniform(x_range[0], x_range[1], k)
        obst[:, :, 1][bad] = LANES[rng.integers(0, 4, k)]
    offsets = np.linspace(-5.25, 5.25, 8)
    g = np.zeros((S, B, 3))
    if goals == "grid":
        assert B % 8 == 0
        g[:, :, 0] = np.tile(offsets, (S, B // 8))
    else:
        g[:, :, 0] = offsets[rng.integers(0, 8, (S, B))]
    g[:, :, 1] = rng.uniform(5.0, 30.0, (S, B))
    return ego, obst, g
