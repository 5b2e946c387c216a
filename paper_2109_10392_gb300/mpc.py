"""Closed-loop MPC on a synthetic highway (the harness around the batch optimizer).

Each cycle (Sec. III intro, Sec. III-F, Sec. IV):
  1. goals are sampled for the driving task (Sec. III-F "Goal Sampling and
     Meta-Cost"): cruise -- goals on every lane at the cruise speed; high-speed
     right-lane -- about 60 % of the goals on the right lane at different
     speeds, the rest spread over the other lanes at the maximum speed;
  2. the neighbours are predicted at constant velocity from their current
     state (Sec. III assumption 3) -- the optimizer does this internally from
     (x0, y0, vx, vy);
  3. the batch is solved (Algorithm 1) and scored (meta cost + heading
     restriction), and the lowest-cost trajectory is taken;
  4. the first dt of that trajectory is executed: the ego advances along it,
     and its controls are read off it (Sec. II: acceleration = dv/dt, steering
     = arctan(psidot h / v), h the inter-axle distance);
  5. the neighbours advance at their own constant velocity (this synthetic
     traffic stands in for the paper's IDM and NGSIM traffic, Sec. IV, which
     are not available) and the frame is shifted so the ego is at x = 0.

The optimizer and the scoring run on the GPU through the C ABI (`mmpc`); the
trajectory sampling of the executed step uses the same Bernstein basis rows
the library builds (mmpc_build), evaluated on the host in FP64.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import mmpc, scenes

CRUISE = "cruise"
HSRL = "hsrl"


@dataclass
class MpcConfig:
    task: str = CRUISE
    v_cruise: float = 20.0     # cruise speed [m/s] (Eq. cruise_cost)
    v_max_goal: float = 25.0   # maximum speed for the high-speed task (Eq. hsrl_cost)
    goals: int = 11            # batch size l (Sec. IV uses 11)
    right_share: float = 0.6   # share of goals on the right lane (high-speed task)
    dt: float = 0.1            # executed part of each plan [s]
    wheelbase: float = 2.7     # inter-axle distance h [m]
    w1: float = 1.0
    w2: float = 0.25
    psi_max_deg: float = 13.0  # heading restriction (Sec. III assumption 2)
    params: dict = field(default_factory=lambda: dict(scenes.BASE_PARAMS))


def sample_goals(cfg: MpcConfig, rng: np.random.Generator) -> np.ndarray:
    """Goal tuples (y_g, v_g, a_g) for one cycle (Sec. III-F)."""
    B = cfg.goals
    lanes = scenes.LANES
    if cfg.task == CRUISE:
        # every lane at the cruise speed, the rest at nearby speeds
        out = []
        k = 0
        while len(out) < B:
            y = lanes[k % len(lanes)]
            dv = 0.0 if k < len(lanes) else float(rng.uniform(-3.0, 3.0))
            out.append((y, cfg.v_cruise + dv, 0.0))
            k += 1
        return np.array(out[:B])
    n_right = int(round(cfg.right_share * B))
    right = np.stack([np.full(n_right, lanes[0]), rng.uniform(0.6, 1.0, n_right) * cfg.v_max_goal,
                      np.zeros(n_right)], 1)
    other_lanes = rng.choice(lanes[1:], B - n_right)
    rest = np.stack([other_lanes, np.full(B - n_right, cfg.v_max_goal), np.zeros(B - n_right)], 1)
    return np.concatenate([right, rest])


def meta_for(cfg: MpcConfig) -> dict:
    if cfg.task == CRUISE:
        return dict(kind=mmpc.MMPC_META_CRUISE, w1=cfg.w1, w2=0.0, v_ref=cfg.v_cruise, y_ref=0.0,
                    psi_max_deg=cfg.psi_max_deg)
    return dict(kind=mmpc.MMPC_META_HSRL, w1=cfg.w1, w2=cfg.w2, v_ref=cfg.v_max_goal, y_ref=float(scenes.LANES[0]),
                psi_max_deg=cfg.psi_max_deg)


class Basis:
    """Bernstein rows of the horizon at arbitrary times (for executing dt):
    de Casteljau evaluation, as in the library's builder."""

    def __init__(self, T: float, n: int):
        self.T, self.n = T, n

    def rows(self, t: float):
        p = self.n - 1
        tau = min(max(t / self.T, 0.0), 1.0)

        def bern(q):
            b = [1.0]
            for _ in range(q):
                nb = [0.0] * (len(b) + 1)
                for k, v in enumerate(b):
                    nb[k] += (1.0 - tau) * v
                    nb[k + 1] += tau * v
                b = nb
            return b

        def get(b, k):
            return b[k] if 0 <= k < len(b) else 0.0
        bp, b1, b2 = bern(p), bern(p - 1), bern(p - 2)
        P = np.array(bp)
        Pd = np.array([p / self.T * (get(b1, k - 1) - get(b1, k)) for k in range(self.n)])
        Pdd = np.array([p * (p - 1) / self.T ** 2 * (get(b2, k - 2) - 2 * get(b2, k - 1) + get(b2, k))
                        for k in range(self.n)])
        return P, Pd, Pdd


def execute(coef: np.ndarray, basis: Basis, dt: float, wheelbase: float):
    """State after dt along a trajectory (c_x, c_y, c_psi) and the controls at
    t = 0: acceleration dv/dt and steering arctan(psidot h / v) (Sec. II)."""
    n = basis.n
    cx, cy, cp = coef[:n], coef[n:2 * n], coef[2 * n:]
    P, Pd, Pdd = basis.rows(dt)
    x, y, psi = P @ cx, P @ cy, P @ cp
    xd, yd = Pd @ cx, Pd @ cy
    v = math.hypot(xd, yd)
    acc = (xd * (Pdd @ cx) + yd * (Pdd @ cy)) / max(v, 1e-6)  # dv/dt
    P0, Pd0, Pdd0 = basis.rows(0.0)
    v0 = math.hypot(Pd0 @ cx, Pd0 @ cy)
    psidot0 = Pd0 @ cp
    steer = math.atan(psidot0 * wheelbase / max(v0, 1e-6))
    acc0 = ((Pd0 @ cx) * (Pdd0 @ cx) + (Pd0 @ cy) * (Pdd0 @ cy)) / max(v0, 1e-6)
    return dict(x=x, y=y, psi=psi, v=v, acc=acc, steer=steer, acc_cmd=acc0)


@dataclass
class CycleLog:
    latency_ms: float
    argmin: int
    cost: float
    ego: np.ndarray
    controls: tuple
    min_clearance: float  # smallest ellipse-normalised distance to a neighbour at the new state


class ClosedLoop:
    """Runs the MPC loop on the GPU for a scene of m neighbours."""

    def __init__(self, cfg: MpcConfig, ego: np.ndarray, obst: np.ndarray, seed: int = 0):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.params = dict(cfg.params)
        self.ego = np.array(ego, dtype=np.float64)
        self.obst = np.array(obst, dtype=np.float64).reshape(-1, 4)
        self.rng = np.random.default_rng(seed)
        self.solver = mmpc.Solver(self.params, self.obst.shape[0])
        self.basis = Basis(self.params["T"], self.params["n"])
        self.meta = mmpc.make_meta(**meta_for(cfg))
        self.dev = torch.device("cuda:0")
        self.warm = None

    def close(self):
        self.solver.close()

    def step(self) -> CycleLog:
        torch = self.torch
        goals = sample_goals(self.cfg, self.rng)
        t0 = time.perf_counter()
        f = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=self.dev)  # noqa: E731
        res = self.solver.solve(f(self.ego), f(self.obst), f(goals), want_lam=False)
        cost, am = self.solver.score(self.meta, res.coef)
        coef = res.coef.double().cpu().numpy()
        cost = cost.cpu().numpy()
        am = int(am.item())
        latency = (time.perf_counter() - t0) * 1e3
        if am < 0:  # every trajectory rejected: keep the one with the smallest heading excursion
            am = 0
        st = execute(coef[am], self.basis, self.cfg.dt, self.cfg.wheelbase)
        dt = self.cfg.dt
        # neighbours move at constant velocity; shift the frame to the ego's new x
        self.obst[:, 0] += self.obst[:, 2] * dt - st["x"]
        self.obst[:, 1] += self.obst[:, 3] * dt
        self.ego = np.array([st["y"], st["v"], st["psi"], st["acc"]])
        a, b = self.params["a"], self.params["b"]
        clear = float(np.min(np.hypot(self.obst[:, 0] / a, (self.obst[:, 1] - st["y"]) / b))) if len(self.obst) else np.inf
        return CycleLog(latency, am, float(cost[am]), self.ego.copy(), (st["acc_cmd"], st["steer"]), clear)

    def run(self, cycles: int) -> list[CycleLog]:
        return [self.step() for _ in range(cycles)]


def summarize(logs: list[CycleLog]) -> dict:
    lat = np.array([l.latency_ms for l in logs])
    return dict(cycles=len(logs), latency_ms_p50=float(np.percentile(lat, 50)),
                latency_ms_p99=float(np.percentile(lat, 99)), solves_per_s=float(1e3 / lat.mean()),
                min_clearance=float(min(l.min_clearance for l in logs)),
                mean_speed=float(np.mean([l.ego[1] for l in logs])),
                final_lane_y=float(logs[-1].ego[0]))
