"""Writes tests/golden/oracle_highway_B11_m10_seed0.json from the FP64 oracle
alone (no CUDA code is imported).  The paper prints no worked example, so this
file is a regression record of the oracle on the 11-goal, 10-obstacle highway
scene (seed 0), not an independent pin.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2109_10392_gb300 import scenes  # noqa: E402


def main():
    sc = scenes.scene_small(0)
    p = oracle.params(**sc.params)
    r = oracle.solve(p, sc.ego, sc.obst, sc.goals)
    meta = sc.meta
    cost, am = oracle.meta_cost(p, r["coef"], kind=meta["kind"], w1=meta["w1"], w2=meta["w2"],
                                v_ref=meta["v_ref"], y_ref=meta["y_ref"], psi_max=np.deg2rad(meta["psi_max_deg"]))
    out = dict(scene="scene_small(seed=0)", params=sc.params, meta=meta,
               ego=sc.ego.tolist(), obst=sc.obst.tolist(), goals=sc.goals.tolist(),
               coef=r["coef"].tolist(), resid=r["resid"].tolist(),
               cost=[c if np.isfinite(c) else "inf" for c in cost.tolist()], argmin=int(am))
    with open(os.path.join(HERE, "oracle_highway_B11_m10_seed0.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
