"""Regression of the oracle against its recorded output on the 11-goal,
10-obstacle highway scene (tests/golden/make_golden.py writes the record
from the oracle alone).  Catches any unintended change of the oracle's
arithmetic; the tolerance covers libm differences between hosts."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_record(orc):
    with open(os.path.join(HERE, "golden", "oracle_highway_B11_m10_seed0.json")) as f:
        g = json.load(f)
    p = orc.params(**g["params"])
    r = orc.solve(p, np.array(g["ego"]), np.array(g["obst"]), np.array(g["goals"]))
    assert np.allclose(r["coef"], np.array(g["coef"]), rtol=1e-7, atol=1e-7)
    m = g["meta"]
    cost, am = orc.meta_cost(p, r["coef"], kind=m["kind"], w1=m["w1"], w2=m["w2"], v_ref=m["v_ref"],
                             y_ref=m["y_ref"], psi_max=np.deg2rad(m["psi_max_deg"]))
    ref = np.array([np.inf if c == "inf" else c for c in g["cost"]])
    assert np.allclose(cost, ref, rtol=1e-9)
    assert am == g["argmin"]
